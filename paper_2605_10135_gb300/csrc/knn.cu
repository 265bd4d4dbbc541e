// Exact per-shard kNN (Sec. IV Workflow (2): each shard's graph is built
// independently, with no exchange between shards).
//
// Distance tiles are dense contractions on the 5th-generation tensor cores:
//   dist(i, j) = |x_i|^2 + |y_j|^2 - 2 x_i . y_j
// The row term |x_i|^2 is constant along a row, so rows are ranked by
// key(i, j) = |y_j|^2 - 2 x_i . y_j and |x_i|^2 is added back at the end.
//
// Kernel k_knn_tiles: one CTA per 128-row block of one problem (a shard, or a
// query batch against all vectors).  Warp roles:
//   warp 0   : TMA producer.  The CTA's A rows (all K) are loaded once and stay
//              in shared memory; B tiles of 256 rows x 64 K-elements stream
//              through an NST-stage ring (128-byte swizzle).
//   warp 1   : allocates 512 TMEM columns (two 128x256 FP32 accumulators) and
//              issues tcgen05.mma (M=128, N=256, K=16) from one thread.
//   warps 2-5: epilogue, one thread per row (TMEM lane).  Each 32-column chunk
//              is read with tcgen05.ld, turned into keys, reduced to a chunk
//              minimum and skipped unless it beats the row's current k-th key;
//              survivors replace the root of a per-row max-heap in shared
//              memory (composite (key, column) order, so ties go to the
//              smaller column = smaller global id).
// Every wait is bounded; on a timeout the CTA records DEV_TIMEOUT, drains its
// copies, frees TMEM and returns.
//
// Operand modes:
//   plain : A = B = one BF16/FP16 copy of the vectors.  uint8 values and their
//           products/sums up to 2^24 are exact in BF16 x BF16 -> FP32, so the
//           integer keys are exact (d <= 258).
//   split : float vectors stored as hi = bf16(x), lo = bf16(x - hi) in two
//           K sections; x.y ~ hi.hi + hi.lo + lo.hi (three products), used to
//           screen a widened list that k_rerank re-scores in FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "stages.cuh"

namespace ann {

namespace kt {
constexpr int BM = 128;
constexpr int BN = 256;
constexpr int KB = 64;                      // K elements per 128-byte block
constexpr int A_BLK_BYTES = BM * 128;       // 16 KB
constexpr int B_BLK_BYTES = BN * 128;       // 32 KB
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr int MAX_NST = 6;
}  // namespace kt

struct KnnParams {
    const int64_t* blk_off;  // [nprob+1] prefix sums of row blocks
    const KnnProblem* probs;
    int nprob;
    const float* nb;  // key bias per B row: |y|^2
    const float* na;  // |x|^2 per A row
    const uint32_t* members;  // column -> global id (NULL: identity)
    int self_exclude;
    int mode;      // 0 plain, 1 split
    int nkb_a;     // resident A k-blocks
    int nkb_b;     // B k-blocks per tile
    int kprime;    // heap entries per row
    int k_out;     // entries written per row
    int nst;       // pipeline stages
    uint32_t idesc;
    uint32_t* out_id;
    float* out_d;
    int* status;
};

struct KnnSmemLayout {
    uint32_t a, b, heap, scratch, bars, tmem_slot, abort_flag, total;
};

__host__ __device__ inline KnnSmemLayout knn_smem_layout(int nkb_a, int nst, int kprime) {
    KnnSmemLayout L;
    uint32_t o = 0;
    L.a = o;
    o += nkb_a * kt::A_BLK_BYTES;
    L.b = o;
    o += nst * kt::B_BLK_BYTES;
    L.heap = o;
    o += kprime * kt::BM * 8;
    L.scratch = o;
    o += kt::BM * 128;
    L.bars = o;
    o += (2 * kt::MAX_NST + 6) * 8;
    L.tmem_slot = o;
    o += 4;
    L.abort_flag = o;
    o += 4;
    L.total = o + 1024;  // slack for 1024-byte alignment of the base
    return L;
}

__device__ __forceinline__ uint64_t heap_init_val() {
    return ((uint64_t)f2ord(INFINITY) << 32) | 0xFFFFFFFFull;
}

// Replace the root of the max-heap of `row` (entries strided by BM) by x and sift down.
__device__ __forceinline__ void heap_replace_root(uint64_t* H, int row, int n, uint64_t x) {
    int e = 0;
    for (;;) {
        int l = 2 * e + 1;
        if (l >= n) break;
        uint64_t hl = H[l * kt::BM + row];
        int c = l;
        uint64_t hc = hl;
        if (l + 1 < n) {
            uint64_t hr = H[(l + 1) * kt::BM + row];
            if (hr > hl) { c = l + 1; hc = hr; }
        }
        if (hc <= x) break;
        H[e * kt::BM + row] = hc;
        e = c;
    }
    H[e * kt::BM + row] = x;
}

__device__ __forceinline__ void heap_sift(uint64_t* H, int row, int e, int n) {
    uint64_t x = H[e * kt::BM + row];
    for (;;) {
        int l = 2 * e + 1;
        if (l >= n) break;
        uint64_t hl = H[l * kt::BM + row];
        int c = l;
        uint64_t hc = hl;
        if (l + 1 < n) {
            uint64_t hr = H[(l + 1) * kt::BM + row];
            if (hr > hl) { c = l + 1; hc = hr; }
        }
        if (hc <= x) break;
        H[e * kt::BM + row] = hc;
        e = c;
    }
    H[e * kt::BM + row] = x;
}

__global__ void __launch_bounds__(kt::THREADS, 1)
    k_knn_tiles(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const KnnParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // Find this CTA's problem and row block.
    const int64_t bid = blockIdx.x;
    if (bid >= P.blk_off[P.nprob]) return;
    int lo = 0, hi = P.nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.blk_off[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    const KnnProblem pr = P.probs[lo];
    const int rb = (int)(bid - P.blk_off[lo]);
    const int ntiles = (pr.n_cols + kt::BN - 1) / kt::BN;

    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const KnnSmemLayout L = knn_smem_layout(P.nkb_a, P.nst, P.kprime);
    const uint32_t sA = smem_u32(base + L.a);
    const uint32_t sB = smem_u32(base + L.b);
    uint64_t* H = (uint64_t*)(base + L.heap);
    float* scratch = (float*)(base + L.scratch);
    const uint32_t bars = smem_u32(base + L.bars);
    const uint32_t full_bar = bars, empty_bar = bars + kt::MAX_NST * 8;
    const uint32_t accf_bar = bars + 2 * kt::MAX_NST * 8, acce_bar = accf_bar + 16;
    const uint32_t a_bar = acce_bar + 16, done_bar = a_bar + 8;
    volatile uint32_t* tmem_slot = (volatile uint32_t*)(base + L.tmem_slot);
    volatile int* abort_flag = (volatile int*)(base + L.abort_flag);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.nst; ++s) {
            mbar_init(full_bar + 8 * s, 1);
            mbar_init(empty_bar + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf_bar + 8 * a, 1);
            mbar_init(acce_bar + 8 * a, 4);
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
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            tma_prefetch_desc(&tmA);
            tma_prefetch_desc(&tmB);
            const int a_y = (int)(pr.a_row0 + (int64_t)rb * kt::BM);
            mbar_expect_tx(a_bar, P.nkb_a * kt::A_BLK_BYTES);
            for (int b = 0; b < P.nkb_a; ++b)
                tma_load_2d(sA + b * kt::A_BLK_BYTES, &tmA, a_bar, b * kt::KB, a_y);
            uint32_t last_par = 0;   // parity of the last load per stage (bit s)
            uint32_t used = 0;       // stages ever loaded (bit s)
            int st = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int t = 0; t < ntiles && ok; ++t) {
                const int b_y = (int)(pr.b_row0 + (int64_t)t * kt::BN);
                for (int j = 0; j < P.nkb_b; ++j) {
                    if (!mbar_wait(empty_bar + 8 * st, ph ^ 1, abort_flag)) { ok = false; break; }
                    mbar_expect_tx(full_bar + 8 * st, kt::B_BLK_BYTES);
                    tma_load_2d(sB + st * kt::B_BLK_BYTES, &tmB, full_bar + 8 * st, j * kt::KB, b_y);
                    used |= 1u << st;
                    last_par = (last_par & ~(1u << st)) | (ph << st);
                    if (++st == P.nst) { st = 0; ph ^= 1; }
                }
            }
            // Drain: every issued copy must land before the CTA may exit.
            int dummy = 0;
            for (int s = 0; s < P.nst; ++s)
                if (used >> s & 1) mbar_wait(full_bar + 8 * s, (last_par >> s) & 1, &dummy, 200000000ull);
            mbar_wait(a_bar, 0, &dummy, 200000000ull);
            if (!ok) atomicOr(P.status, DEV_TIMEOUT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------- MMA
        if (lane == 0) {
            bool ok = mbar_wait(a_bar, 0, abort_flag);
            tc_fence_after();
            int st = 0;
            uint32_t ph = 0;
            const int H2 = P.nkb_b >> 1;
            for (int t = 0; t < ntiles && ok; ++t) {
                const int a = t & 1;
                if (!mbar_wait(acce_bar + 8 * a, ((t >> 1) & 1) ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem + a * kt::BN;
                uint32_t accum = 0;
                for (int j = 0; j < P.nkb_b; ++j) {
                    if (!mbar_wait(full_bar + 8 * st, ph, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t bsm = sB + st * kt::B_BLK_BYTES;
                    // A blocks paired with this B block.
                    int ablk[2];
                    int na = 1;
                    if (P.mode == 0) {
                        ablk[0] = j;
                    } else if (j < H2) {
                        ablk[0] = j;        // hi.hi
                        ablk[1] = H2 + j;   // lo.hi
                        na = 2;
                    } else {
                        ablk[0] = j - H2;   // hi.lo
                    }
                    for (int q = 0; q < na; ++q) {
                        const uint32_t asm_ = sA + ablk[q] * kt::A_BLK_BYTES;
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            umma_f16(d_tmem, sdesc_sw128(asm_ + s * 32), sdesc_sw128(bsm + s * 32),
                                     P.idesc, accum);
                            accum = 1;
                        }
                    }
                    umma_commit(empty_bar + 8 * st);
                    if (++st == P.nst) { st = 0; ph ^= 1; }
                }
                if (!ok) break;
                umma_commit(accf_bar + 8 * a);
            }
            // Wait for every issued MMA before TMEM is released.
            umma_commit(done_bar);
            int dummy = 0;
            mbar_wait(done_bar, 0, &dummy, 200000000ull);
            if (!ok) atomicOr(P.status, DEV_TIMEOUT);
        }
    } else {
        // -------------------------------------------------------- epilogue
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int row = q * 32 + lane;
        const int i = rb * kt::BM + row;  // row index inside the problem
        const int kp = P.kprime;
        const uint64_t init = heap_init_val();
        for (int e = 0; e < kp; ++e) H[e * kt::BM + row] = init;
        float tau = INFINITY;
        const float* nbp = P.nb + pr.b_row0;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        float* scr = scratch + row;  // element u at scr[u * BM]: conflict-free
        bool ok = true;
        for (int t = 0; t < ntiles; ++t) {
            const int a = t & 1;
            if (!mbar_wait(accf_bar + 8 * a, (t >> 1) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            for (int c = 0; c < kt::BN / 32; ++c) {
                const int j0 = t * kt::BN + c * 32;
                uint32_t v[32];
                __syncwarp();
                tmem_ld32(tmem + lane_addr + a * kt::BN + c * 32, v);
                tmem_wait_ld();
                if (j0 >= pr.n_cols) continue;  // uniform over the warp
                float key[32];
                const float4* nb4 = (const float4*)(nbp + j0);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float4 nn = __ldg(nb4 + u);
                    key[4 * u + 0] = fmaf(-2.0f, __uint_as_float(v[4 * u + 0]), nn.x);
                    key[4 * u + 1] = fmaf(-2.0f, __uint_as_float(v[4 * u + 1]), nn.y);
                    key[4 * u + 2] = fmaf(-2.0f, __uint_as_float(v[4 * u + 2]), nn.z);
                    key[4 * u + 3] = fmaf(-2.0f, __uint_as_float(v[4 * u + 3]), nn.w);
                }
                const bool edge = (j0 + 32 > pr.n_cols) ||
                                  (P.self_exclude && (unsigned)(i - j0) < 32u);
                if (edge) {
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int j = j0 + u;
                        if (j >= pr.n_cols || (P.self_exclude && j == i)) key[u] = INFINITY;
                    }
                }
                float m = key[0];
#pragma unroll
                for (int u = 1; u < 32; ++u) m = fminf(m, key[u]);
                if (!__any_sync(0xffffffffu, m < tau)) continue;
                uint32_t bits = 0;
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    bits |= (key[u] < tau ? 1u : 0u) << u;
                    scr[u * kt::BM] = key[u];
                }
                while (__any_sync(0xffffffffu, bits != 0)) {
                    if (bits) {
                        const int u = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const float kv = scr[u * kt::BM];
                        if (kv < tau) {
                            const uint64_t x = ((uint64_t)f2ord(kv) << 32) | (uint32_t)(j0 + u);
                            heap_replace_root(H, row, kp, x);
                            tau = ord2f((uint32_t)(H[row] >> 32));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar + 8 * a);
        }
        if (!ok) {
            atomicOr(P.status, DEV_TIMEOUT);
        } else if (i < pr.n_rows) {
            // Heap sort ascending, then write (global id, |x|^2 + key).
            for (int end = kp - 1; end > 0; --end) {
                uint64_t top = H[row];
                H[row] = H[end * kt::BM + row];
                H[end * kt::BM + row] = top;
                heap_sift(H, row, 0, end);
            }
            const float nx = P.na[pr.a_row0 + i];
            const int64_t orow = pr.out_row0 + i;
            for (int e = 0; e < P.k_out; ++e) {
                const uint64_t x = H[e * kt::BM + row];
                const uint32_t j = (uint32_t)x;
                uint32_t id = ANN_PAD;
                float dd = INFINITY;
                if (j != 0xFFFFFFFFu) {
                    id = P.members ? __ldg(P.members + pr.mem_row0 + j) : j;
                    dd = nx + ord2f((uint32_t)(x >> 32));
                }
                P.out_id[orow * P.k_out + e] = id;
                P.out_d[orow * P.k_out + e] = dd;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kt::TMEM_COLS);
    }
}

// ---- problem tables, gather and norms ------------------------------------------
// probs[s] for the C shards: a/b rows at the 128-padded offsets, out rows at offsets.
__global__ void k_shard_tables(const int64_t* __restrict__ offsets, int C, int64_t rows,
                               int64_t* __restrict__ blk_off, int64_t* __restrict__ pad_off,
                               KnnProblem* __restrict__ probs, int* status) {
    if (threadIdx.x || blockIdx.x) return;
    int64_t b = 0, p = 0;
    bool bad = offsets[0] != 0 || offsets[C] != rows;
    for (int s = 0; s < C; ++s) {
        int64_t n = offsets[s + 1] - offsets[s];
        if (n < 0 || n >= (1ll << 24)) { bad = true; n = 0; }
        blk_off[s] = b;
        pad_off[s] = p;
        KnnProblem pr;
        pr.a_row0 = p;
        pr.b_row0 = p;
        pr.out_row0 = offsets[s];
        pr.mem_row0 = offsets[s];
        pr.n_rows = (int32_t)n;
        pr.n_cols = (int32_t)n;
        probs[s] = pr;
        int64_t nbk = (n + kt::BM - 1) / kt::BM;
        b += nbk;
        p += nbk * kt::BM;
    }
    blk_off[C] = bad ? 0 : b;  // nothing runs on inconsistent input
    pad_off[C] = p;
    if (bad) atomicOr(status, DEV_BAD_INPUT);
}

// Gather rows into the tile layout: row p' of G (pitch Kp elements) holds the
// operand copy of member (pad_off -> shard, local index) or zeros.
// mode 0: Kp >= d, element t = cvt(x_t).  mode 1: [hi | lo] sections of Kh each.
template <typename T>
__device__ __forceinline__ T cvt_from_float(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_float(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half cvt_from_float(float v) { return __float2half_rn(v); }

template <typename T>
__global__ void k_gather(const void* X, int dtype, int d, const uint32_t* __restrict__ members,
                         const int64_t* __restrict__ offsets, const int64_t* __restrict__ pad_off,
                         int C, int64_t rows_cap, int mode, int Kp, int Kh, T* __restrict__ G,
                         float* __restrict__ norms) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t pr = warp_g; pr < rows_cap; pr += nwarps) {
        int64_t src = -1;
        if (pr < pad_off[C]) {
            int lo = 0, hi = C - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (pad_off[mid] <= pr) lo = mid; else hi = mid - 1;
            }
            int64_t li = pr - pad_off[lo];
            if (li < offsets[lo + 1] - offsets[lo]) {
                int64_t p = offsets[lo] + li;
                src = members ? (int64_t)members[p] : p;
            }
        }
        T* g = G + pr * Kp;
        float nrm = 0.0f;
        for (int t = lane; t < Kp; t += 32) {
            float v = 0.0f;
            if (mode == 0) {
                if (src >= 0 && t < d) {
                    v = load_elem(X, dtype, src * d + t);
                    nrm = fmaf(v, v, nrm);
                }
                g[t] = cvt_from_float<T>(v);
            } else {
                int tt = t < Kh ? t : t - Kh;
                T out = cvt_from_float<T>(0.0f);
                if (src >= 0 && tt < d) {
                    v = load_elem(X, dtype, src * d + tt);
                    T h = cvt_from_float<T>(v);
                    if (t < Kh) {
                        out = h;
                        nrm = fmaf(v, v, nrm);
                    } else {
                        out = cvt_from_float<T>(v - (float)h);
                    }
                }
                g[t] = out;
            }
        }
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if (lane == 0) norms[pr] = nrm;
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
                    uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v[e], lp);
                    uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v[e] >> 32), lp);
                    uint64_t o = ((uint64_t)hi << 32) | lo;
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

template <int E>
__global__ void k_rerank(const void* X, const void* Xrow, int dtype, int d,
                         const uint32_t* __restrict__ row_ids, int64_t nrows,
                         const uint32_t* __restrict__ cand, int kc, int k,
                         uint32_t* __restrict__ out_id, float* __restrict__ out_d) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= nrows) return;
    const int64_t u = row_ids ? (int64_t)row_ids[p] : p;
    uint64_t keys[E];
#pragma unroll
    for (int e = 0; e < E; ++e) keys[e] = ~0ull;
    for (int c = 0; c < kc; ++c) {
        const uint32_t v = cand[p * kc + c];
        if (v == ANN_PAD) continue;  // uniform
        float s = 0.0f;
        for (int t = lane; t < d; t += 32) {
            float df = __fsub_rn(load_elem(Xrow, dtype, u * d + t), load_elem(X, dtype, (int64_t)v * d + t));
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

static int make_tmap(CUtensorMap* m, const void* G, int64_t rows, int Kp, int box_rows) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return fail(ANN_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)G, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ANN_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ANN_OK;
}

int knn_plan(int d, int dtype, int k, int rerank_k, KnnPlan* pl) {
    KnnPlan p;
    if (dtype == ANN_F32) {
        p.mode = 1;
        p.Kh = (int)align_up((size_t)d, kt::KB);
        p.Kp = 2 * p.Kh;
        p.ab_fmt = 1;
        p.rerank = true;
    } else {
        p.mode = 0;
        p.Kh = 0;
        p.Kp = (int)align_up((size_t)d, kt::KB);
        p.ab_fmt = dtype == ANN_F16 ? 0 : 1;
        p.rerank = dtype != ANN_U8;
    }
    p.nkb_a = p.Kp / kt::KB;
    p.nkb_b = p.nkb_a;
    p.kprime = p.rerank ? (rerank_k > 0 ? rerank_k : k + 16) : k;
    if (p.kprime < k) p.kprime = k;
    if (p.rerank && p.kprime > 128) return fail(ANN_ERR_UNSUPPORTED, "re-rank width > 128");
    // Stages: as many as fit (2 .. MAX_NST).
    const size_t cap = 227 * 1024;
    p.nst = 0;
    for (int nst = kt::MAX_NST; nst >= 2; --nst) {
        if (knn_smem_layout(p.nkb_a, nst, p.kprime).total <= cap) { p.nst = nst; break; }
    }
    if (!p.nst)
        return fail(ANN_ERR_UNSUPPORTED, "shard_knn: d=%d with k'=%d does not fit shared memory", d,
                    p.kprime);
    p.smem = knn_smem_layout(p.nkb_a, p.nst, p.kprime).total;
    *pl = p;
    return ANN_OK;
}

size_t knn_ws(int C, int64_t rows, const KnnPlan& pl, KnnWs* out, void* base, size_t cap) {
    Carver cv(base, cap);
    KnnWs w;
    w.rows_cap = rows + (int64_t)kt::BM * C + kt::BN;
    w.blk_off = cv.take<int64_t>(C + 1);
    w.pad_off = cv.take<int64_t>(C + 1);
    w.probs = cv.take<KnnProblem>(C);
    w.G = cv.take<__nv_bfloat16>((size_t)w.rows_cap * pl.Kp);
    w.norms = cv.take<float>((size_t)w.rows_cap + 512);
    w.cand_id = pl.rerank ? cv.take<uint32_t>((size_t)rows * pl.kprime) : nullptr;
    w.cand_d = pl.rerank ? cv.take<float>((size_t)rows * pl.kprime) : nullptr;
    if (out) *out = w;
    return cv.used + 256;
}

static int launch_tiles(const KnnPlan& pl, const void* GA, int64_t rowsA, const void* GB,
                        int64_t rowsB, const KnnParams& P, int64_t grid, cudaStream_t st) {
    CUtensorMap ta, tb;
    int rc = make_tmap(&ta, GA, rowsA, pl.Kp, kt::BM);
    if (rc) return rc;
    rc = make_tmap(&tb, GB, rowsB, pl.Kp, kt::BN);
    if (rc) return rc;
    ANN_CHECK_CUDA(cudaFuncSetAttribute(k_knn_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)pl.smem));
    if (grid <= 0) return ANN_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (tile_timing_on()) {
        e0 = tile_event();
        e1 = tile_event();
        ANN_CHECK_CUDA(cudaEventRecord(e0, st));
    }
    k_knn_tiles<<<(unsigned)grid, kt::THREADS, pl.smem, st>>>(ta, tb, P);
    ANN_CHECK_LAUNCH();
    if (e0) {
        ANN_CHECK_CUDA(cudaEventRecord(e1, st));
        tile_timing_record(e0, e1);
    }
    return ANN_OK;
}

static int launch_rerank(const void* X, const void* Xrow, int dtype, int d, const uint32_t* row_ids,
                         int64_t nrows, const uint32_t* cand, int kc, int k, uint32_t* out_id,
                         float* out_d, cudaStream_t st) {
    const int threads = 128;
    const unsigned grid = (unsigned)((nrows * 32 + threads - 1) / threads);
    if (nrows == 0) return ANN_OK;
    if (kc <= 64)
        k_rerank<2><<<grid, threads, 0, st>>>(X, Xrow, dtype, d, row_ids, nrows, cand, kc, k, out_id, out_d);
    else
        k_rerank<4><<<grid, threads, 0, st>>>(X, Xrow, dtype, d, row_ids, nrows, cand, kc, k, out_id, out_d);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

int run_shard_knn(const void* X, int64_t N, int d, int dtype, const uint32_t* members,
                  const int64_t* offsets, int C, int64_t rows, int k, const KnnPlan& pl,
                  const KnnWs& w, uint32_t* knn_id, float* knn_d, cudaStream_t st) {
    (void)N;
    k_shard_tables<<<1, 32, 0, st>>>(offsets, C, rows, w.blk_off, w.pad_off, w.probs,
                                     device_status_ptr());
    ANN_CHECK_LAUNCH();
    {
        const int threads = 256;
        int64_t want = (w.rows_cap * 32 + threads - 1) / threads;
        unsigned grid = (unsigned)(want < 152 * 64 ? want : 152 * 64);
        if (pl.ab_fmt == 1)
            k_gather<__nv_bfloat16><<<grid, threads, 0, st>>>(X, dtype, d, members, offsets, w.pad_off,
                                                              C, w.rows_cap, pl.mode, pl.Kp, pl.Kh,
                                                              w.G, w.norms);
        else
            k_gather<__half><<<grid, threads, 0, st>>>(X, dtype, d, members, offsets, w.pad_off, C,
                                                      w.rows_cap, pl.mode, pl.Kp, pl.Kh,
                                                      (__half*)w.G, w.norms);
        ANN_CHECK_LAUNCH();
    }
    KnnParams P;
    P.blk_off = w.blk_off;
    P.probs = w.probs;
    P.nprob = C;
    P.nb = w.norms;
    P.na = w.norms;
    P.members = members;
    P.self_exclude = 1;
    P.mode = pl.mode;
    P.nkb_a = pl.nkb_a;
    P.nkb_b = pl.nkb_b;
    P.kprime = pl.kprime;
    P.k_out = pl.rerank ? pl.kprime : k;
    P.nst = pl.nst;
    P.idesc = idesc_f16(kt::BM, kt::BN, pl.ab_fmt);
    P.out_id = pl.rerank ? w.cand_id : knn_id;
    P.out_d = pl.rerank ? w.cand_d : knn_d;
    P.status = device_status_ptr();
    const int64_t grid = rows / kt::BM + C + 1;  // upper bound on row blocks
    int rc = launch_tiles(pl, w.G, w.rows_cap, w.G, w.rows_cap, P, grid, st);
    if (rc) return rc;
    if (pl.rerank)
        return launch_rerank(X, X, dtype, d, members, rows, w.cand_id, pl.kprime, k, knn_id,
                             knn_d, st);
    return ANN_OK;
}

// Query side: A = queries, B = all N vectors (one problem, no self exclusion).
size_t query_ws(int64_t N, int64_t nq, const KnnPlan& pl, QueryWs* out, void* base, size_t cap) {
    Carver cv(base, cap);
    QueryWs w;
    w.capA = nq + kt::BM + kt::BN;
    w.capB = N + kt::BM + kt::BN;
    w.blk_off = cv.take<int64_t>(4);
    w.pad_off = cv.take<int64_t>(4);
    w.offs = cv.take<int64_t>(4);
    w.prob = cv.take<KnnProblem>(1);
    w.GA = cv.take<__nv_bfloat16>((size_t)w.capA * pl.Kp);
    w.GB = cv.take<__nv_bfloat16>((size_t)w.capB * pl.Kp);
    w.na = cv.take<float>((size_t)w.capA + 512);
    w.nb = cv.take<float>((size_t)w.capB + 512);
    w.cand_id = pl.rerank ? cv.take<uint32_t>((size_t)nq * pl.kprime) : nullptr;
    w.cand_d = pl.rerank ? cv.take<float>((size_t)nq * pl.kprime) : nullptr;
    if (out) *out = w;
    return cv.used + 256;
}

__global__ void k_query_tables(int64_t N, int64_t nq, int64_t* blk_off, int64_t* pad4,
                               int64_t* offs4, KnnProblem* prob) {
    if (threadIdx.x || blockIdx.x) return;
    blk_off[0] = 0;
    blk_off[1] = (nq + kt::BM - 1) / kt::BM;
    offs4[0] = 0;   // A side (queries): offsets {0, nq}, padded {0, nq rounded up}
    offs4[1] = nq;
    offs4[2] = 0;   // B side (all vectors): offsets {0, N}
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
    const int threads = 256;
    auto grid_for = [&](int64_t rows_cap) {
        int64_t want = (rows_cap * 32 + threads - 1) / threads;
        return (unsigned)(want < 152 * 64 ? want : 152 * 64);
    };
    if (pl.ab_fmt == 1) {
        k_gather<__nv_bfloat16><<<grid_for(w.capA), threads, 0, st>>>(
            Q, dtype, d, nullptr, w.offs, w.pad_off, 1, w.capA, pl.mode, pl.Kp, pl.Kh, w.GA, w.na);
        k_gather<__nv_bfloat16><<<grid_for(w.capB), threads, 0, st>>>(
            X, dtype, d, nullptr, w.offs + 2, w.pad_off + 2, 1, w.capB, pl.mode, pl.Kp, pl.Kh, w.GB,
            w.nb);
    } else {
        k_gather<__half><<<grid_for(w.capA), threads, 0, st>>>(
            Q, dtype, d, nullptr, w.offs, w.pad_off, 1, w.capA, pl.mode, pl.Kp, pl.Kh,
            (__half*)w.GA, w.na);
        k_gather<__half><<<grid_for(w.capB), threads, 0, st>>>(
            X, dtype, d, nullptr, w.offs + 2, w.pad_off + 2, 1, w.capB, pl.mode, pl.Kp, pl.Kh,
            (__half*)w.GB, w.nb);
    }
    ANN_CHECK_LAUNCH();
    KnnParams P;
    P.blk_off = w.blk_off;
    P.probs = w.prob;
    P.nprob = 1;
    P.nb = w.nb;
    P.na = w.na;
    P.members = nullptr;
    P.self_exclude = 0;
    P.mode = pl.mode;
    P.nkb_a = pl.nkb_a;
    P.nkb_b = pl.nkb_b;
    P.kprime = pl.kprime;
    P.k_out = pl.rerank ? pl.kprime : k;
    P.nst = pl.nst;
    P.idesc = idesc_f16(kt::BM, kt::BN, pl.ab_fmt);
    P.out_id = pl.rerank ? w.cand_id : out_id;
    P.out_d = pl.rerank ? w.cand_d : out_d;
    P.status = device_status_ptr();
    const int64_t grid = (nq + kt::BM - 1) / kt::BM;
    int rc = launch_tiles(pl, w.GA, w.capA, w.GB, w.capB, P, grid, st);
    if (rc) return rc;
    if (pl.rerank)
        return launch_rerank(X, Q, dtype, d, nullptr, nq, w.cand_id, pl.kprime, k, out_id, out_d, st);
    return ANN_OK;
}

}  // namespace ann
