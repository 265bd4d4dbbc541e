// Prune (intermediate degree L = k to final degree R; Sec. III and Sec. VI-B2
// use L = 2R) and merge of the replicated shard graphs by edge union (Sec. II-B,
// Sec. IV Workflow (3)).
//
// Prune, one warp per shard row u: u's list goes into an id -> position table
// in shared memory (one probe per lookup, a multiplier chosen per row so that
// no two of its ids share a slot); the lists of u's neighbours are read with
// coalesced warp loads, every entry looked up, and the counts c_j kept in
// registers (a warp OR-reduction per neighbour).  The R entries of smallest
// (c_j, j) are chosen by a warp bitonic sort and written in list order with a
// ballot/popc compaction.  Integer logic only.
//
// Merge, one warp per vector g: its pruned lists (one per shard holding g) are
// gathered, sorted by (id, distance) to drop duplicate ids (the smaller
// distance survives), re-sorted by (distance, id), and the first R written.
// A variant merge adds reverse edges to a merged graph (k_merge_rev).
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

// Position of id x in the row's list: a direct-mapped table of TS slots.  The
// multiplicative hash y = x * A (A odd) is a bijection of 32-bit words, so the
// slot (the top 10 bits of y) and the low 22 bits of y identify x; one 32-bit
// word per slot holds those 22 bits (bits 10..31) and the position (bits 0..9),
// so a probe's word XOR (y << 10) is the position when the slot holds x and at
// least 1023 otherwise (an empty slot holds all ones).
// For each row the warp tries multipliers until none of the row's ids share a
// slot (about one try in seven succeeds for 64 ids in 1,024 slots); then every
// lookup is one probe.  A row for which no multiplier is found within PTRY tries
// (and every list wider than 64) keeps the colliding ids in a short overflow
// list, scanned when a lookup's slot holds another id.
constexpr int TS = 1024, TSHIFT = 22;  // 2^(32 - TSHIFT) = TS slots
constexpr uint32_t HM = 2654435761u, TEMPTY = 0xFFFFFFFFu;
constexpr int PTRY = 32;

__device__ __forceinline__ uint32_t tmult(int a) { return HM + 0x3C6EF372u * (uint32_t)a; }  // odd
__device__ __forceinline__ uint32_t tkey(uint32_t y) { return y << 10; }  // low 22 bits << 10

// Shared memory of one prune warp: table words [TS], overflow ids and positions
// [KM each], the neighbours' rows [KM], the overflow count (+pad).
__host__ __device__ constexpr size_t prune_warp_smem(int KM) {
    return (size_t)TS * 4 + (size_t)KM * 16 + 16;
}

// Detour counts of one row: for each neighbour v_i (i < m) the warp reads L_{v_i}
// with coalesced loads (entry t in lane t % 32, register t / 32) and looks each
// entry up in u's table; an entry at position j of u's list with i < j and t < j
// sets bit j of the lane's mask.  The ids of a list are distinct, so OR over the
// lanes counts each (i, j) pair once; lane l adds bit l of word e to c[e], the
// count of position j = l + 32 e.
template <int E, bool OVF>
__device__ __forceinline__ void prune_counts(const uint32_t* __restrict__ knn_id, int k, int m,
                                             const int64_t* wrow, const uint32_t* tw,
                                             const uint32_t* ovf, const uint32_t* ovf_pos,
                                             int novf, uint32_t A, uint32_t (&c)[E]) {
    constexpr int G = E <= 2 ? 4 : 2;  // neighbour lists read together (loads in flight)
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < m; i0 += G) {
        uint32_t x[G][E];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int i = i0 + g;
            const int64_t w = i < m ? wrow[i] : -1;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int t = lane + 32 * e;
                x[g][e] = (w >= 0 && t < k) ? __ldg(knn_id + w * k + t) : ANN_PAD;
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int i = i0 + g;
            if (i >= m) break;  // warp-uniform
            // (ANN_PAD entries never match: the table holds only the row's ids)
            uint32_t bits[E];
            uint64_t bits64 = 0;  // E <= 2: positions 0..63 in one word
#pragma unroll
            for (int e = 0; e < E; ++e) bits[e] = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int t = lane + 32 * e;
                const uint32_t thr = (uint32_t)(i > t ? i : t);  // hit: thr < j < 256
                const uint32_t y = x[g][e] * A;
                const uint32_t wd = tw[y >> TSHIFT];
                uint32_t dj = wd ^ tkey(y);  // the position j when the slot holds x
                if (OVF && dj >= 256u && wd != TEMPTY && novf > 0) {
                    for (int o = 0; o < novf; ++o)
                        if (ovf[o] == x[g][e]) dj = ovf_pos[o];
                }
                if (dj - thr - 1u < 255u - thr) {
                    if constexpr (E <= 2) {
                        bits64 |= 1ull << dj;
                    } else {
#pragma unroll
                        for (int e2 = 0; e2 < E; ++e2)
                            if ((int)(dj >> 5) == e2) bits[e2] |= 1u << (dj & 31u);
                    }
                }
            }
            if constexpr (E <= 2) {
                bits[0] = (uint32_t)bits64;
                if (E == 2) bits[E - 1] = (uint32_t)(bits64 >> 32);
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (32 * e + 31 <= i) continue;  // no j > i in this word (uniform)
                c[e] += (__reduce_or_sync(0xffffffffu, bits[e]) >> lane) & 1u;
            }
        }
    }
}

// One warp per shard row u, lists of width k <= 32 E; entry j of u's list (j =
// lane + 32 e) sits in lane `lane`, register e.  The counts c_j of the
// rank-based detour prune (Sec. III; CAGRA's rule), then the R positions of
// smallest (c_j, j) kept in list order.
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
    uint32_t* tw = (uint32_t*)my;                  // [TS]
    int64_t* wrow = (int64_t*)(tw + TS);           // [KM]
    uint32_t* ovf = (uint32_t*)(wrow + KM);        // [KM]
    uint32_t* ovf_pos = ovf + KM;                  // [KM]
    int* novf_p = (int*)(ovf_pos + KM);            // [1] (+pad)
    const uint32_t lt = (1u << lane) - 1;
    // the table starts empty once; after each row only the slots its ids used are
    // emptied again
    for (int h = lane; h < TS; h += 32) tw[h] = TEMPTY;
    __syncwarp();

    for (int64_t p = blockIdx.x * (int64_t)nwb + wib; p < rows; p += (int64_t)gridDim.x * nwb) {
        const int s = shard_of(offsets, C, p);
        const int64_t m0 = __ldg(offsets + s), m1 = __ldg(offsets + s + 1);
        uint32_t lu[E];  // u's list: entry lane + 32 e
        int m = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int t = lane + 32 * e;
            lu[e] = t < k ? __ldg(knn_id + p * k + t) : ANN_PAD;
            m += __popc(__ballot_sync(0xffffffffu, lu[e] != ANN_PAD));
        }
        uint32_t kb[E];  // kept positions: bit j & 31 of word j >> 5, in every lane
#pragma unroll
        for (int e = 0; e < E; ++e) kb[e] = 0;
        if (rule == ANN_PRUNE_TRUNC) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int lim = (R < m ? R : m) - 32 * e;
                kb[e] = lim >= 32 ? 0xFFFFFFFFu : lim > 0 ? (1u << lim) - 1 : 0u;
            }
        } else {
            // the neighbours' rows in this shard (independent loads, all in flight)
            int64_t wr[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = lane + 32 * e;
                wr[e] = j < m ? row_in_range(start, rowlist, lu[e], m0, m1) : -1;
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (lane + 32 * e < m) wrow[lane + 32 * e] = wr[e];
            // a multiplier under which the row's ids occupy distinct slots
            uint32_t A = HM;
            bool perfect = false;
            for (int a = 0; a < (E <= 2 ? PTRY : 0) && !perfect; ++a) {
                A = tmult(a);
                bool clash = false;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int j = lane + 32 * e;
                    if (j < m) {
                        const uint32_t y = lu[e] * A;
                        if (atomicCAS(&tw[y >> TSHIFT], TEMPTY, tkey(y) | (uint32_t)j) != TEMPTY)
                            clash = true;
                    }
                }
                perfect = !__any_sync(0xffffffffu, clash);
                if (!perfect) {  // empty every slot the row's ids touched, try the next
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (lane + 32 * e < m) tw[(lu[e] * A) >> TSHIFT] = TEMPTY;
                    __syncwarp();
                }
            }
            int novf = 0;
            if (!perfect) {  // the table with an overflow list
                A = HM;
                if (lane == 0) *novf_p = 0;
                __syncwarp();
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int j = lane + 32 * e;
                    if (j < m) {
                        const uint32_t y = lu[e] * A;
                        if (atomicCAS(&tw[y >> TSHIFT], TEMPTY, tkey(y) | (uint32_t)j) != TEMPTY) {
                            const int o = atomicAdd(novf_p, 1);
                            ovf[o] = lu[e];
                            ovf_pos[o] = (uint32_t)j;
                        }
                    }
                }
                __syncwarp();
                novf = *novf_p;
            }
            __syncwarp();
            uint32_t c[E];
#pragma unroll
            for (int e = 0; e < E; ++e) c[e] = 0;
            if (novf == 0)
                prune_counts<E, false>(knn_id, k, m, wrow, tw, ovf, ovf_pos, 0, A, c);
            else
                prune_counts<E, true>(knn_id, k, m, wrow, tw, ovf, ovf_pos, novf, A, c);
            // rank positions by (c_j, j); any starting placement sorts the same
            uint32_t sel[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = lane + 32 * e;
                sel[e] = j < m ? ((c[e] << 16) | (uint32_t)j) : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (lane + 32 * e < m) tw[(lu[e] * A) >> TSHIFT] = TEMPTY;
            warp_sort<E, uint32_t>(sel);
            // sel[] (element index lane*E+e) ranks positions; keep the first min(R, m)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int idx = lane * E + e;
                if (idx < R && sel[e] != 0xFFFFFFFFu) {
                    const uint32_t jj = sel[e] & 0xFFFFu;
#pragma unroll
                    for (int e2 = 0; e2 < E; ++e2)
                        if ((int)(jj >> 5) == e2) kb[e2] |= 1u << (jj & 31);
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e) kb[e] = __reduce_or_sync(0xffffffffu, kb[e]);
        }
        // the kept entries in list order
        int outc = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (32 * e >= m) break;
            const int j = lane + 32 * e;
            const bool f = j < m && ((kb[e] >> lane) & 1u);
            const uint32_t b = __ballot_sync(0xffffffffu, f);
            if (f) {
                const int pos = outc + __popc(b & lt);
                pr_id[p * R + pos] = lu[e];
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

// ---- merge with reverse edges (a variant of the merge) ----------------------------
// For every vertex v of a merged graph: the first ceil(R/2) entries of its own
// list, then the vertices u whose lists hold v (edge distance d(u, v)) in
// (distance, id) order, skipping ids already taken, then the rest of its own
// list, up to R entries; the result sorted by (distance, id).  Reverse edges
// are what CAGRA adds after its rank-based prune; the paper merges by edge union
// only (Sec. II-B), so this is an alternative merge, not a step of the method.
__global__ void k_rev_count(const uint32_t* __restrict__ graph, const uint32_t* __restrict__ degree,
                            int64_t N, int R, int32_t* __restrict__ cnt, int* status) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * R;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = q / R;
        const uint32_t du = degree[u];
        if ((int)(q - u * R) >= (int)(du < (uint32_t)R ? du : (uint32_t)R)) continue;
        const uint32_t v = graph[q];
        if (v < N && v != (uint32_t)u) atomicAdd(cnt + v, 1); else atomicOr(status, DEV_BAD_INPUT);
    }
}

// rkey[start[v] ..]: (order bits of d(u, v) << 32 | u) of every edge u -> v, in
// arrival order (the selection below sorts them).
__global__ void k_rev_fill(const uint32_t* __restrict__ graph, const float* __restrict__ gdist,
                           const uint32_t* __restrict__ degree, int64_t N, int R,
                           const int64_t* __restrict__ start, int32_t* __restrict__ fill,
                           uint64_t* __restrict__ rkey) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * R;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = q / R;
        const uint32_t du = degree[u];
        if ((int)(q - u * R) >= (int)(du < (uint32_t)R ? du : (uint32_t)R)) continue;
        const uint32_t v = graph[q];
        if (v >= N || v == (uint32_t)u) continue;
        const int slot = atomicAdd(fill + v, 1);
        rkey[start[v] + slot] = ((uint64_t)f2ord(gdist[q]) << 32) | (uint32_t)u;
    }
}

// One warp per vertex v, R <= 64: own entry j = lane + 32 e in lane `lane`,
// register e; the first half (j < h <= 32) is in register 0 of lanes 0 .. h-1.
// The reverse sources are taken 64 at a time into a shared buffer beside the 64
// best so far and the 128 sorted; the buffer then holds the final list's keys.
constexpr int REV_WARPS = 4;
__global__ void __launch_bounds__(REV_WARPS * 32)
    k_merge_rev(const uint32_t* __restrict__ graph, const float* __restrict__ gdist,
                const uint32_t* __restrict__ degree, const int64_t* __restrict__ start,
                const uint64_t* __restrict__ rkey, int64_t N, int R,
                uint32_t* __restrict__ out_g, float* __restrict__ out_d,
                uint32_t* __restrict__ out_deg) {
    __shared__ uint64_t sbuf[REV_WARPS][128];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t v = blockIdx.x * (int64_t)REV_WARPS + wib;
    if (v >= N) return;  // warp-uniform
    uint64_t* buf = sbuf[wib];
    const uint32_t dg = degree[v];
    const int dv = (int)(dg < (uint32_t)R ? dg : (uint32_t)R);
    uint32_t oid[2];
    uint64_t okey[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int j = lane + 32 * e;
        oid[e] = j < dv ? graph[v * R + j] : ANN_PAD;
        okey[e] = j < dv ? (((uint64_t)f2ord(gdist[v * R + j]) << 32) | oid[e]) : ~0ull;
    }
    const int half = (R + 1) / 2;
    const int h = dv < half ? dv : half;
    const int Q = R - h;
    buf[lane] = ~0ull;
    buf[lane + 32] = ~0ull;
    const int64_t r0 = start[v], r1 = start[v + 1];
    for (int64_t c0 = r0; c0 < r1; c0 += 64) {
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t c = c0 + lane + 32 * e;
            uint64_t key = c < r1 ? rkey[c] : ~0ull;
            const uint32_t src = (uint32_t)key;
            bool dup = false;
            for (int q = 0; q < h; ++q) dup |= __shfl_sync(0xffffffffu, oid[0], q) == src;
            buf[64 + lane + 32 * e] = dup ? ~0ull : key;
        }
        __syncwarp();
        uint64_t k4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) k4[e] = buf[lane * 4 + e];
        warp_sort<4, uint64_t>(k4);
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (lane * 4 + e < 64) buf[lane * 4 + e] = k4[e];
    }
    __syncwarp();
    // the chosen reverse sources: the first nsel (<= Q) of buf[0, 64)
    int nsel = 0;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = lane + 32 * e;
        nsel += __popc(__ballot_sync(0xffffffffu, i < Q && buf[i] != ~0ull));
    }
    // the rest of v's own list (j >= h) that is not among them, in list order
    int left = R - h - nsel;
    bool keep[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int j = lane + 32 * e;
        bool ok = j >= h && j < dv;
        if (ok)
            for (int i = 0; i < nsel; ++i)
                if ((uint32_t)buf[i] == oid[e]) { ok = false; break; }
        keep[e] = ok;
    }
    int nkeep = 0;
    const uint32_t lt = (1u << lane) - 1;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const uint32_t b = __ballot_sync(0xffffffffu, keep[e]);
        const int rank = nkeep + __popc(b & lt);
        keep[e] = keep[e] && rank < left;
        nkeep += __popc(b);
    }
    nkeep = nkeep < left ? nkeep : left;
    // the final keys in buf[64, 128): own first half, then the chosen, then the
    // kept rest (any placement: they are sorted next)
    buf[64 + lane] = ~0ull;
    buf[96 + lane] = ~0ull;
    __syncwarp();
    if (lane < h) buf[64 + lane] = okey[0];
    for (int i = lane; i < nsel; i += 32) buf[64 + h + i] = buf[i];
    {
        int base = h + nsel;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t b = __ballot_sync(0xffffffffu, keep[e]);
            if (keep[e]) buf[64 + base + __popc(b & lt)] = okey[e];
            base += __popc(b);
        }
    }
    __syncwarp();
    uint64_t fk[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) fk[e] = buf[64 + lane * 2 + e];
    warp_sort<2, uint64_t>(fk);
    const int n = h + nsel + nkeep;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int pos = lane * 2 + e;
        if (pos < R) {
            const bool f = pos < n;
            out_g[v * R + pos] = f ? (uint32_t)fk[e] : ANN_PAD;
            out_d[v * R + pos] = f ? ord2f((uint32_t)(fk[e] >> 32)) : INFINITY;
        }
    }
    if (lane == 0) out_deg[v] = (uint32_t)n;
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

size_t merge_rev_ws(int64_t N, int R, MergeRevWs* out, void* base, size_t cap) {
    Carver cv(base, cap);
    MergeRevWs w;
    w.cnt = cv.take<int32_t>((size_t)N + 1);
    w.start = cv.take<int64_t>((size_t)N + 1);
    w.bsum = cv.take<int64_t>((size_t)(N / SCAN_CHUNK + 2));
    w.rkey = cv.take<uint64_t>((size_t)(N * R > 0 ? N * R : 1));
    if (out) *out = w;
    return cv.used + 256;
}

int run_merge_reverse(const uint32_t* graph, const float* gdist, const uint32_t* degree, int64_t N,
                      int R, uint32_t* out_g, float* out_d, uint32_t* out_deg, const MergeRevWs& w,
                      cudaStream_t st) {
    if (N == 0) return ANN_OK;
    const int tpb = 256;
    ANN_CHECK_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * (N + 1), st));
    k_rev_count<<<grid_of(N * R, tpb), tpb, 0, st>>>(graph, degree, N, R, w.cnt,
                                                      device_status_ptr());
    ANN_CHECK_LAUNCH();
    const int64_t nb = (N + SCAN_CHUNK - 1) / SCAN_CHUNK;
    k_scan_sums<<<(unsigned)nb, SCAN_T, 0, st>>>(w.cnt, N, w.bsum);
    ANN_CHECK_LAUNCH();
    k_scan_bsums<<<1, 1024, 0, st>>>(w.bsum, nb);
    ANN_CHECK_LAUNCH();
    k_scan_apply<<<(unsigned)nb, SCAN_T, 0, st>>>(w.cnt, N, w.bsum, w.start);
    ANN_CHECK_LAUNCH();
    ANN_CHECK_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * (N + 1), st));
    k_rev_fill<<<grid_of(N * R, tpb), tpb, 0, st>>>(graph, gdist, degree, N, R, w.start, w.cnt,
                                                     w.rkey);
    ANN_CHECK_LAUNCH();
    k_merge_rev<<<(unsigned)((N + REV_WARPS - 1) / REV_WARPS), REV_WARPS * 32, 0, st>>>(
        graph, gdist, degree, w.start, w.rkey, N, R, out_g, out_d, out_deg);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

}  // namespace ann
