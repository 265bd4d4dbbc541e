// Learned candidate form: a d -> 256 -> 32 projection MLP proposes each shard
// row's candidate neighbours in embedding space; the candidates are re-ranked
// with exact FP32 distances in the original space.  The paper builds shard graphs
// from exact distances only (Sec. II-B, Sec. IV Workflow (2)); this form is an
// addition beside it, measured by its recall against the exact graph.
//
// Model    f(x) = W2 relu(W1 (x / s) + b1) + b2, s = max |x| over all vectors;
//          parameters are one FP32 array [W1 (256 x d) | b1 | W2 (32 x 256) | b2].
// Training triplet margin loss (1/B) sum max(0, |f(a)-f(p)|^2 - |f(a)-f(n)|^2 + m)
//          with Adam (0.9, 0.999, 1e-8, bias-corrected), FP32 master weights.
//          Anchors come from a sample of the vectors; their exact kk nearest
//          vectors (tile query kernel over all N) give positives (first kpos)
//          and near-miss negatives (the rest), half the negatives are uniform
//          rows.  The random picks are caller inputs.
// Kernels  layer 1 (d -> 256) of a training step on the tensor cores: the
//          forward product and the weight gradient dW1 = dU^T (x / s) as
//          tcgen05.mma GEMMs, each FP32 operand (x / s, W1, dU) split into two
//          BF16 parts and multiplied as hi.hi + lo.hi + hi.lo with FP32
//          accumulation (FP32 master weights); the small layer-2 products as
//          FP32 tiled GEMMs (64 x 64 x 16 tiles, every output summed over k in
//          increasing order); the embedding of all rows on the tensor cores
//          (FP16 operands); small element-wise kernels for the loss, Adam and
//          the triplet picks.  Split-K partial products are summed in slice
//          order, so every result is deterministic.
#include "stages.cuh"

namespace ann {

// A matrix operand read element by element: logical (r, c) is stored at row r,
// column c (trans = 0) or row c, column r (trans = 1); the stored row index goes
// through an optional gather map, then row0 is added; the value is converted from
// dtype and multiplied by *sp (a device scalar) when sp is set.
struct Mat {
    const void* p;
    int dtype;
    const uint32_t* gather;
    int64_t row0;
    int64_t ld;
    int trans;
    const float* sp;
};

__device__ __forceinline__ float mat_at(const Mat& m, int64_t r, int64_t c, float s) {
    const int64_t sr = m.trans ? c : r, sc = m.trans ? r : c;
    const int64_t row = (m.gather ? (int64_t)m.gather[sr] : sr) + m.row0;
    return load_elem(m.p, m.dtype, row * m.ld + sc) * s;
}

// C[M x N] = A[M x K] . B[K x N], ep(i, j, acc) stores each output.
template <class EP>
__global__ void __launch_bounds__(256) k_sgemm(int64_t M, int N, int K, Mat A, Mat B, EP ep) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * 64;
    const int n0 = blockIdx.y * 64;
    const float sa = A.sp ? *A.sp : 1.0f, sb = B.sp ? *B.sp : 1.0f;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + q * 256;
            const int r = A.trans ? (e & 63) : (e >> 4);  // consecutive threads follow
            const int c = A.trans ? (e >> 6) : (e & 15);  // the stored rows
            const int64_t gi = m0 + r;
            const int gk = k0 + c;
            As[c][r] = (gi < M && gk < K) ? mat_at(A, gi, gk, sa) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + q * 256;
            const int r = B.trans ? (e & 15) : (e >> 6);
            const int c = B.trans ? (e >> 4) : (e & 63);
            const int gk = k0 + r, gj = n0 + c;
            Bs[r][c] = (gk < K && gj < N) ? mat_at(B, gk, gj, sb) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gi = m0 + ty * 4 + i;
            const int gj = n0 + tx * 4 + j;
            if (gi < M && gj < N) ep(gi, gj, acc[i][j]);
        }
}

// ---- epilogues ---------------------------------------------------------------
struct EpHidden {  // U = acc + b1 (kept for the backward pass if U is set), H = relu(U)
    float* U;
    float* H;
    const float* b;
    int ld;
    __device__ void operator()(int64_t i, int j, float acc) const {
        const float u = acc + b[j];
        if (U) U[i * ld + j] = u;
        H[i * ld + j] = u > 0.0f ? u : 0.0f;
    }
};
struct EpBias {  // C = acc + b
    float* C;
    const float* b;
    int ld;
    __device__ void operator()(int64_t i, int j, float acc) const { C[i * ld + j] = acc + b[j]; }
};
struct EpStore {  // C = acc
    float* C;
    int ld;
    __device__ void operator()(int64_t i, int j, float acc) const { C[i * ld + j] = acc; }
};
struct EpReluMask {  // C = acc where U > 0, else 0 (back through the ReLU)
    float* C;
    const float* U;
    int ld;
    __device__ void operator()(int64_t i, int j, float acc) const {
        C[i * ld + j] = U[i * ld + j] > 0.0f ? acc : 0.0f;
    }
};

// Split-K: slice z of the K range [z * ks, (z + 1) * ks) into part[z][M x N].
struct EpPart {
    float* part;
    int64_t M;
    int N;
    __device__ void operator()(int64_t i, int j, float acc) const { part[i * N + j] = acc; }
};

__global__ void __launch_bounds__(256)
    k_sgemm_split(int64_t M, int N, int K, int kslice, Mat A, Mat B, float* part) {
    // shift the K window of this slice into the operands' row / column offsets
    const int z = blockIdx.z;
    const int k0 = z * kslice;
    const int kn = K - k0 < kslice ? K - k0 : kslice;
    Mat a = A, b = B;
    // A is logical M x K: K is its column (trans 0) or stored row (trans 1)
    if (a.trans) {
        if (a.gather) a.gather += k0; else a.row0 += k0;
    } else {
        a.p = (const char*)a.p + (int64_t)k0 * (a.dtype == ANN_F32 ? 4 : (a.dtype == ANN_U8 ? 1 : 2));
    }
    // B is logical K x N: K is its stored row (trans 0) or column (trans 1)
    if (!b.trans) {
        if (b.gather) b.gather += k0; else b.row0 += k0;
    } else {
        b.p = (const char*)b.p + (int64_t)k0 * (b.dtype == ANN_F32 ? 4 : (b.dtype == ANN_U8 ? 1 : 2));
    }
    EpPart ep{part + (int64_t)z * M * N, M, N};
    // same tile loop as k_sgemm on the slice
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * 64;
    const int n0 = blockIdx.y * 64;
    const float sa = a.sp ? *a.sp : 1.0f, sb = b.sp ? *b.sp : 1.0f;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int kk0 = 0; kk0 < kn; kk0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + q * 256;
            const int r = a.trans ? (e & 63) : (e >> 4);
            const int c = a.trans ? (e >> 6) : (e & 15);
            const int64_t gi = m0 + r;
            const int gk = kk0 + c;
            As[c][r] = (gi < M && gk < kn) ? mat_at(a, gi, gk, sa) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = t + q * 256;
            const int r = b.trans ? (e & 15) : (e >> 6);
            const int c = b.trans ? (e >> 4) : (e & 63);
            const int gk = kk0 + r, gj = n0 + c;
            Bs[r][c] = (gk < kn && gj < N) ? mat_at(b, gk, gj, sb) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gi = m0 + ty * 4 + i;
            const int gj = n0 + tx * 4 + j;
            if (gi < M && gj < N) ep(gi, gj, acc[i][j]);
        }
}

// Sum of the slices in slice order, then the real epilogue.
template <class EP>
__global__ void k_split_reduce(const float* __restrict__ part, int nz, int64_t M, int N, EP ep) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= M * N) return;
    float s = 0.0f;
    for (int z = 0; z < nz; ++z) s += part[(int64_t)z * M * N + q];
    ep(q / N, (int)(q % N), s);
}

// Grids that would leave most of the 152 SMs idle with long K loops (the weight
// gradients: M x N small, K = 3 x batch) are split along K into slices whose
// partial products are summed in slice order; part must hold nz * M * N floats.
static constexpr int64_t SPLIT_PART_FLOATS = (int64_t)1 << 22;

template <class EP>
static int gemm(int64_t M, int N, int K, const Mat& A, const Mat& B, const EP& ep,
                cudaStream_t st, float* part = nullptr) {
    if (M <= 0 || N <= 0) return ANN_OK;
    const dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64));
    const int64_t blocks = (int64_t)grid.x * grid.y;
    int nz = 1;
    if (part && blocks < 304 && K >= 256) {
        nz = (int)((304 + blocks - 1) / blocks);
        if (nz > K / 64) nz = K / 64;
        while (nz > 1 && (int64_t)nz * M * N > SPLIT_PART_FLOATS) --nz;
    }
    if (nz <= 1) {
        k_sgemm<EP><<<grid, 256, 0, st>>>(M, N, K, A, B, ep);
        ANN_CHECK_LAUNCH();
        return ANN_OK;
    }
    int kslice = (K + nz - 1) / nz;
    kslice = (kslice + 15) / 16 * 16;
    nz = (K + kslice - 1) / kslice;
    k_sgemm_split<<<dim3(grid.x, grid.y, nz), 256, 0, st>>>(M, N, K, kslice, A, B, part);
    ANN_CHECK_LAUNCH();
    k_split_reduce<EP><<<(unsigned)((M * N + 255) / 256), 256, 0, st>>>(part, nz, M, N, ep);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

static Mat mat(const void* p, int dtype, int64_t ld, int trans = 0, const uint32_t* gather = nullptr,
               int64_t row0 = 0, const float* sp = nullptr) {
    Mat m;
    m.p = p;
    m.dtype = dtype;
    m.gather = gather;
    m.row0 = row0;
    m.ld = ld;
    m.trans = trans;
    m.sp = sp;
    return m;
}

// ---- tensor-core GEMM of the training step ------------------------------------
// D[M x N] (FP32) = A[M x K] . B[N x K]^T, BF16 operands stored K-major with rows
// padded to whole tiles (missing rows of the tensor map read as zeros) and K a
// multiple of 64.  One 128 x 256 output tile per CTA, the K blocks of slice
// blockIdx.z: warp 0 issues TMA copies into a ring of 3 stages, warp 1 the
// tcgen05.mma (FP32 accumulator in TMEM), then every warp reads its 32 rows
// back (thread = row) and hands ep(row, col, value, slice) each output.
namespace tgm {
constexpr int BM = 128, BN = 256, KB = 64, NST = 3;
constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128, STAGE = A_BYTES + B_BYTES;
constexpr int THREADS = 128;
constexpr size_t SMEM = 1024 + (size_t)NST * STAGE + (2 * NST + 1) * 8 + 16;
}  // namespace tgm

template <class EP>
__global__ void __launch_bounds__(tgm::THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int64_t M, int N, int nkb, int kb_per_slice, uint32_t idesc, EP ep, int* status) {
    using namespace tgm;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t ring = smem_u32(base);
    uint8_t* tail = base + NST * STAGE;
    const uint32_t bars = smem_u32(tail);
    const uint32_t full = bars, empty = bars + NST * 8, done = bars + 2 * NST * 8;
    volatile uint32_t* tslot = (volatile uint32_t*)(tail + (2 * NST + 1) * 8);
    volatile int* abort_flag = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kb_per_slice;
    const int kb1 = kb0 + kb_per_slice < nkb ? kb0 + kb_per_slice : nkb;
    if (threadIdx.x == 0) {
        for (int st = 0; st < NST; ++st) {
            mbar_init(full + 8 * st, 1);
            mbar_init(empty + 8 * st, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32((const void*)tslot), BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        uint32_t used = 0, last_par = 0;
        for (int kb = kb0; kb < kb1; ++kb) {
            const int i = kb - kb0, st = i % NST;
            const uint32_t ph = (uint32_t)(i / NST) & 1u;
            if (!mbar_wait(empty + 8 * st, ph ^ 1u, abort_flag)) { ok = false; break; }
            mbar_expect_tx(full + 8 * st, STAGE);
            tma_load_2d(ring + st * STAGE, &tmA, full + 8 * st, kb * KB, (int)m0);
            tma_load_2d(ring + st * STAGE + A_BYTES, &tmB, full + 8 * st, kb * KB, n0);
            used |= 1u << st;
            last_par = (last_par & ~(1u << st)) | (ph << st);
        }
        int dummy = 0;  // every issued copy lands before the CTA may exit
        for (int st = 0; st < NST; ++st)
            if (used >> st & 1) mbar_wait(full + 8 * st, (last_par >> st) & 1u, &dummy, 200000000ull);
        if (!ok) atomicOr(status, DEV_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        for (int kb = kb0; kb < kb1; ++kb) {
            const int i = kb - kb0, st = i % NST;
            const uint32_t ph = (uint32_t)(i / NST) & 1u;
            if (!mbar_wait(full + 8 * st, ph, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a = ring + st * STAGE, b = a + A_BYTES;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                umma_f16(tmem, sdesc_sw128(a + q * 32), sdesc_sw128(b + q * 32), idesc,
                         (i | q) != 0 ? 1u : 0u);
            umma_commit(empty + 8 * st);
        }
        umma_commit(done);  // also after a timeout: every issued MMA completes first
        if (!ok) atomicOr(status, DEV_TIMEOUT);
    }
    __syncwarp();
    const bool got = mbar_wait(done, 0, abort_flag);
    tc_fence_after();
    if (got && !*abort_flag) {
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t v[32];
            tmem_ld32(tmem + lane_addr + c * 32, v);
            tmem_wait_ld();
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + c * 32 + j;
                    if (col < N) ep(row, col, __uint_as_float(v[j]), (int)blockIdx.z);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(status, DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

struct EpTcHidden {  // U = acc + b1, H = relu(U), row-major with ld columns
    float* U;
    float* H;
    const float* b;
    int ld;
    __device__ void operator()(int64_t i, int j, float acc, int) const {
        const float u = acc + b[j];
        U[i * ld + j] = u;
        H[i * ld + j] = u > 0.0f ? u : 0.0f;
    }
};
struct EpTcPart {  // slice z's partial output part[z][M x N]
    float* part;
    int64_t M;
    int N;
    __device__ void operator()(int64_t i, int j, float acc, int z) const {
        part[((int64_t)z * M + i) * N + j] = acc;
    }
};

// Layer 1's FP32 operands go to the tensor cores as two BF16 parts, hi = bf16(v)
// and lo = bf16(v - hi), laid out along K so that one BF16 GEMM over 3 K sums
// hi.hi + lo.hi + hi.lo (the lo.lo term, below 2^-16 of the product, is dropped).
// Batch rows x / s: row-major [Rp x 3Kp] as [hi | lo | hi] and transposed
// [Kp x 3Rp] as [hi | hi | lo] (zeros past R rows and d columns).
__device__ __forceinline__ void bf16_split(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}
__global__ void k_batch_bf16(const void* X, int dtype, int d, const uint32_t* __restrict__ idx,
                             int64_t R, int64_t Rp, int Kp, const float* __restrict__ inv_s,
                             __nv_bfloat16* __restrict__ rows, __nv_bfloat16* __restrict__ cols) {
    const float sc = *inv_s;
    const int64_t tot = Rp * Kp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / Kp;
        const int t = (int)(q - r * Kp);
        const float v = (r < R && t < d) ? load_elem(X, dtype, (int64_t)idx[r] * d + t) * sc : 0.0f;
        __nv_bfloat16 hi, lo;
        bf16_split(v, hi, lo);
        __nv_bfloat16* rw = rows + r * 3 * Kp + t;
        rw[0] = hi;
        rw[Kp] = lo;
        rw[2 * Kp] = hi;
        __nv_bfloat16* cl = cols + (int64_t)t * 3 * Rp + r;
        cl[0] = hi;
        cl[Rp] = hi;
        cl[2 * Rp] = lo;
    }
}

// W1 [256 x d] FP32 -> [256 x 3Kp] as [hi | hi | lo]; dU [R x 256] FP32 ->
// transposed [256 x 3Rp] as [hi | lo | hi].
__global__ void k_w1_bf16(const float* __restrict__ W1, int d, int Kp,
                          __nv_bfloat16* __restrict__ out) {
    const int64_t tot = (int64_t)ml::HID * Kp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = q / Kp;
        const int t = (int)(q - h * Kp);
        __nv_bfloat16 hi, lo;
        bf16_split(t < d ? W1[h * d + t] : 0.0f, hi, lo);
        __nv_bfloat16* o = out + h * 3 * Kp + t;
        o[0] = hi;
        o[Kp] = hi;
        o[2 * Kp] = lo;
    }
}
__global__ void k_du_bf16_t(const float* __restrict__ dU, int64_t R, int64_t Rp,
                            __nv_bfloat16* __restrict__ out) {
    const int64_t tot = (int64_t)ml::HID * Rp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = q / Rp, r = q - h * Rp;
        __nv_bfloat16 hi, lo;
        bf16_split(r < R ? dU[r * ml::HID + h] : 0.0f, hi, lo);
        __nv_bfloat16* o = out + h * 3 * Rp + r;
        o[0] = hi;
        o[Rp] = lo;
        o[2 * Rp] = hi;
    }
}

template <class EP>
static int gemm_tc(const void* A, int64_t rowsA, const void* B, int64_t rowsB, int Kp, int64_t M,
                   int N, int nz, const EP& ep, cudaStream_t st) {
    CUtensorMap ta, tb;
    int rc = make_tmap(&ta, A, rowsA, Kp, tgm::KB, tgm::BM, CU_TENSOR_MAP_SWIZZLE_128B);
    if (!rc) rc = make_tmap(&tb, B, rowsB, Kp, tgm::KB, tgm::BN, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    ANN_CHECK_CUDA(cudaFuncSetAttribute(k_gemm_tc<EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tgm::SMEM));
    const int nkb = Kp / tgm::KB;
    const int per = (nkb + nz - 1) / nz;
    const dim3 grid((unsigned)((M + tgm::BM - 1) / tgm::BM), (unsigned)((N + tgm::BN - 1) / tgm::BN),
                    (unsigned)((nkb + per - 1) / per));
    k_gemm_tc<EP><<<grid, tgm::THREADS, tgm::SMEM, st>>>(ta, tb, M, N, nkb, per,
                                                         idesc_f16(tgm::BM, tgm::BN, 1), ep,
                                                         device_status_ptr());
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

// ---- small kernels -----------------------------------------------------------
// 1 / max|x| (1 when every element is 0).
__global__ void k_inv_scale(const unsigned int* amax_bits, float* inv) {
    if (threadIdx.x || blockIdx.x) return;
    const float a = __uint_as_float(*amax_bits);
    *inv = a > 0.0f ? __frcp_rn(a) : 1.0f;
}

// Triplet rows of one step: idx[i] = anchor, idx[B + i] = positive, idx[2B + i] =
// negative, from draws [B x 3] (anchor slot, r1, r2).
// Ids at or above N (bad input) are replaced by 0 and reported in the status word.
__device__ __forceinline__ uint32_t safe_id(uint32_t v, int64_t N, int* status) {
    if ((int64_t)v < N) return v;
    atomicOr(status, DEV_BAD_INPUT);
    return 0;
}

__global__ void k_triplets(const uint32_t* __restrict__ sample, int64_t S,
                           const uint32_t* __restrict__ knn, int kk, int kpos,
                           const uint32_t* __restrict__ draws, const int* __restrict__ step,
                           int B, int64_t N, uint32_t* __restrict__ idx, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint32_t* dr = draws + ((int64_t)*step * B + i) * 3;
    const int64_t j = (int64_t)(dr[0] % (uint64_t)S);
    const uint32_t* L = knn + j * kk;
    const uint32_t r2 = dr[2];
    idx[i] = safe_id(sample[j], N, status);
    idx[B + i] = safe_id(L[dr[1] % (uint32_t)kpos], N, status);
    idx[2 * B + i] = (r2 & 1u) ? (uint32_t)((uint64_t)(r2 >> 1) % (uint64_t)N)
                               : safe_id(L[kpos + (r2 >> 1) % (uint32_t)(kk - kpos)], N, status);
}

// Per triplet: loss term and the gradient of the batch loss w.r.t. the three
// embeddings (rows i, B + i, 2B + i of Z / dZ).
__global__ void k_triplet_loss(const float* __restrict__ Z, int B, float margin,
                               float* __restrict__ dZ, float* __restrict__ li) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const float* za = Z + (int64_t)i * ml::OUT;
    const float* zp = Z + (int64_t)(B + i) * ml::OUT;
    const float* zn = Z + (int64_t)(2 * B + i) * ml::OUT;
    float dp = 0.0f, dn = 0.0f;
    for (int c = 0; c < ml::OUT; ++c) {
        const float u = za[c] - zp[c], v = za[c] - zn[c];
        dp = fmaf(u, u, dp);
        dn = fmaf(v, v, dn);
    }
    const float h = dp - dn + margin;
    const bool act = h > 0.0f;
    li[i] = act ? h : 0.0f;
    const float g = act ? 2.0f / (float)B : 0.0f;
    float* ga = dZ + (int64_t)i * ml::OUT;
    float* gp = dZ + (int64_t)(B + i) * ml::OUT;
    float* gn = dZ + (int64_t)(2 * B + i) * ml::OUT;
    for (int c = 0; c < ml::OUT; ++c) {
        ga[c] = g * (zn[c] - zp[c]);
        gp[c] = g * (zp[c] - za[c]);
        gn[c] = g * (za[c] - zn[c]);
    }
}

// out[j] = sum over rows of A[row * cols + j], rows in increasing order.
__global__ void k_colsum(const float* __restrict__ A, int64_t rows, int cols,
                         float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.0f;
    for (int64_t r = 0; r < rows; ++r) s += A[r * cols + j];
    out[j] = s;
}

// Mean of li[0..B) into out[*step] (fixed tree order, one block).
__global__ void k_mean(const float* __restrict__ li, int B, const int* __restrict__ step,
                       float* out) {
    __shared__ float red[256];
    float s = 0.0f;
    for (int i = threadIdx.x; i < B; i += 256) s += li[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[*step] = red[0] / (float)B;
}

// One Adam step on n parameters, t = *step + 1; c1 = 1 / (1 - beta1^t),
// c2 = 1 / (1 - beta2^t) (in double, rounded once).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, const int* __restrict__ step) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = (double)(*step + 1);
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, t)));
    const float c2 = (float)(1.0 / (1.0 - pow(0.999, t)));
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

__global__ void k_step_advance(int* step) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ++*step;
}

// Copy rows sample[j] of X (esize bytes per element) into Q row j.
__global__ void k_gather_rows(const uint8_t* __restrict__ X, int64_t row_bytes,
                              const uint32_t* __restrict__ rows, int64_t n, int64_t N,
                              uint8_t* __restrict__ Q, int* status) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const uint8_t* s = X + (int64_t)safe_id(rows[w], N, status) * row_bytes;
    uint8_t* q = Q + w * row_bytes;
    for (int64_t b = lane; b < row_bytes; b += 32) q[b] = s[b];
}

// The kk nearest other vectors of sample row j: its kk+1 list without itself
// (without the last entry if the row itself is not listed).
__global__ void k_drop_self(const uint32_t* __restrict__ ids, int kq,
                            const uint32_t* __restrict__ sample, int64_t S,
                            uint32_t* __restrict__ knn) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= S) return;
    const uint32_t self = sample[j];
    int o = 0;
    for (int e = 0; e < kq && o < kq - 1; ++e) {
        const uint32_t v = ids[j * kq + e];
        if (v != self) knn[j * (kq - 1) + o++] = v;
    }
    for (; o < kq - 1; ++o) knn[j * (kq - 1) + o] = ANN_PAD;
}

// hits += |truth[j][0..tk) intersect found[j][0..fk)| over rows j.
__global__ void k_cover(const uint32_t* __restrict__ found, int fs, int fk,
                        const uint32_t* __restrict__ truth, int ts, int tk, int64_t n,
                        unsigned long long* hits) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long h = 0;
    if (j < n) {
        for (int a = 0; a < tk; ++a) {
            const uint32_t t = truth[j * ts + a];
            if (t == ANN_PAD) continue;
            for (int b = 0; b < fk; ++b)
                if (found[j * fs + b] == t) {
                    ++h;
                    break;
                }
        }
    }
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0 && h) atomicAdd(hits, h);
}

__global__ void k_hits_to_recall(const unsigned long long* hits, int64_t denom, float* out) {
    if (threadIdx.x || blockIdx.x) return;
    *out = denom > 0 ? (float)((double)*hits / (double)denom) : 0.0f;
}

// ---- embedding of all rows on the tensor cores ------------------------------------
// Layer 1 (x/s . W1^T, K = d) runs as tcgen05.mma (M=128, N=256, K=16) on FP16
// operands: the scaled inputs lie in [-1, 1] and the weights are small, so FP16
// keeps 11 significant bits where BF16 would keep 8.  One CTA per 128 rows: warp 0
// feeds a 3-stage TMA ring (the rows' 64-element K block and W1's), warp 1 issues
// the MMAs into 256 TMEM columns, then all four warps read their 32 rows back,
// add b1, apply ReLU and do layer 2 (256 -> 32) in FP32 from shared memory.
namespace emb {
constexpr int BM = 128;
constexpr int KB = 64;
constexpr int NST = 3;
constexpr int A_BYTES = BM * 128;
constexpr int B_BYTES = ml::HID * 128;
constexpr int STAGE = A_BYTES + B_BYTES;
constexpr int THREADS = 128;
constexpr int W2T_FLOATS = ml::HID * ml::OUT;
constexpr size_t SMEM = 1024 + (size_t)NST * STAGE + (size_t)(W2T_FLOATS + ml::HID + ml::OUT) * 4 +
                        (2 * NST + 1) * 8 + 16;
}  // namespace emb

__global__ void __launch_bounds__(emb::THREADS, 1)
    k_embed_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
               int64_t n, int nkb, uint32_t idesc, const float* __restrict__ b1,
               const float* __restrict__ W2, const float* __restrict__ b2, float* __restrict__ E,
               int* status) {
    using namespace emb;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t ring = smem_u32(base);
    float* w2t = (float*)(base + NST * STAGE);  // [h][o]
    float* sb1 = w2t + W2T_FLOATS;
    float* sb2 = sb1 + ml::HID;
    uint8_t* tail = (uint8_t*)(sb2 + ml::OUT);
    const uint32_t bars = smem_u32(tail);
    const uint32_t full = bars, empty = bars + NST * 8, done = bars + 2 * NST * 8;
    volatile uint32_t* tslot = (volatile uint32_t*)(tail + (2 * NST + 1) * 8);
    volatile int* abort_flag = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(full + 8 * s, 1);
            mbar_init(empty + 8 * s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32((const void*)tslot), ml::HID);
        tmem_relinquish();
    }
    for (int i = threadIdx.x; i < W2T_FLOATS; i += THREADS)
        w2t[i] = W2[(i % ml::OUT) * ml::HID + i / ml::OUT];
    for (int i = threadIdx.x; i < ml::HID; i += THREADS) sb1[i] = b1[i];
    if (threadIdx.x < ml::OUT) sb2[threadIdx.x] = b2[threadIdx.x];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;
    if (warp == 0 && lane == 0) {
        // producer
        tma_prefetch_desc(&tmX);
        tma_prefetch_desc(&tmW);
        uint32_t used = 0, last_par = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % NST;
            const uint32_t ph = (uint32_t)(kb / NST) & 1u;
            if (!mbar_wait(empty + 8 * s, ph ^ 1u, abort_flag)) { ok = false; break; }
            mbar_expect_tx(full + 8 * s, STAGE);
            tma_load_2d(ring + s * STAGE, &tmX, full + 8 * s, kb * KB, (int)row0);
            tma_load_2d(ring + s * STAGE + A_BYTES, &tmW, full + 8 * s, kb * KB, 0);
            used |= 1u << s;
            last_par = (last_par & ~(1u << s)) | (ph << s);
        }
        int dummy = 0;  // every issued copy lands before the CTA may exit
        for (int s = 0; s < NST; ++s)
            if (used >> s & 1) mbar_wait(full + 8 * s, (last_par >> s) & 1u, &dummy, 200000000ull);
        if (!ok) atomicOr(status, DEV_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        // MMA issue
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % NST;
            const uint32_t ph = (uint32_t)(kb / NST) & 1u;
            if (!mbar_wait(full + 8 * s, ph, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a = ring + s * STAGE, b = a + A_BYTES;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                umma_f16(tmem, sdesc_sw128(a + q * 32), sdesc_sw128(b + q * 32), idesc,
                         (kb | q) != 0 ? 1u : 0u);
            umma_commit(empty + 8 * s);
        }
        umma_commit(done);  // also after a timeout: every issued MMA completes first
        if (!ok) atomicOr(status, DEV_TIMEOUT);
    }
    __syncwarp();
    // epilogue: thread = row (TMEM lane)
    const bool got = mbar_wait(done, 0, abort_flag);
    tc_fence_after();
    if (got && !*abort_flag) {
        float z[ml::OUT];
#pragma unroll
        for (int o = 0; o < ml::OUT; ++o) z[o] = sb2[o];
        const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
        for (int c = 0; c < ml::HID / 32; ++c) {
            uint32_t v[32];
            tmem_ld32(tmem + lane_addr + c * 32, v);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int h = c * 32 + j;
                float hv = __uint_as_float(v[j]) + sb1[h];
                hv = hv > 0.0f ? hv : 0.0f;
                const float4* w = (const float4*)(w2t + h * ml::OUT);
#pragma unroll
                for (int q = 0; q < ml::OUT / 4; ++q) {
                    const float4 ww = w[q];
                    z[4 * q] = fmaf(hv, ww.x, z[4 * q]);
                    z[4 * q + 1] = fmaf(hv, ww.y, z[4 * q + 1]);
                    z[4 * q + 2] = fmaf(hv, ww.z, z[4 * q + 2]);
                    z[4 * q + 3] = fmaf(hv, ww.w, z[4 * q + 3]);
                }
            }
        }
        const int64_t row = row0 + warp * 32 + lane;
        if (row < n) {
            float4* out = (float4*)(E + row * ml::OUT);
#pragma unroll
            for (int q = 0; q < ml::OUT / 4; ++q)
                out[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
        }
    } else if (threadIdx.x == 0) {
        atomicOr(status, DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, ml::HID);
    }
}

// FP16 operands: out[i][t] = half(in(row r0 + i, t) * scale) for i < n and t < d,
// 0 elsewhere (rows up to n_pad, columns up to Kp).
__global__ void k_to_half_rows(const void* X, int dtype, int d, int64_t r0, int64_t n,
                               int64_t n_pad, int Kp, const float* __restrict__ inv_s,
                               __half* __restrict__ out) {
    const float sc = inv_s ? *inv_s : 1.0f;
    const int64_t total = n_pad * Kp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / Kp;
        const int t = (int)(q - i * Kp);
        out[q] = __float2half_rn(i < n && t < d ? load_elem(X, dtype, (r0 + i) * d + t) * sc
                                                : 0.0f);
    }
}

static constexpr int64_t EMB_CHUNK = 65536;

static int64_t emb_chunk(int d) {
    const int64_t Kp = (d + emb::KB - 1) / emb::KB * emb::KB;
    int64_t ch = ((int64_t)256 << 20) / (Kp * 2);  // at most 256 MB of FP16 rows
    if (ch > EMB_CHUNK) ch = EMB_CHUNK;
    return ch / emb::BM * emb::BM > 0 ? ch / emb::BM * emb::BM : emb::BM;
}

// Rows of one embedding launch, rounded up to whole 128-row blocks.
static int64_t emb_rows_buf(int64_t N, int d) {
    const int64_t ch = N < emb_chunk(d) ? N : emb_chunk(d);
    return (ch + emb::BM - 1) / emb::BM * emb::BM > 0 ? (ch + emb::BM - 1) / emb::BM * emb::BM
                                                      : emb::BM;
}

size_t learned_embed_ws(int64_t N, int d) {
    const int64_t Kp = (d + emb::KB - 1) / emb::KB * emb::KB;
    Carver cv(nullptr, ~(size_t)0);
    cv.take<unsigned int>(4);
    cv.take<float>(4);
    cv.take<__half>((size_t)emb_rows_buf(N, d) * Kp);
    cv.take<__half>((size_t)ml::HID * Kp);
    return cv.used + 256;
}

int run_learned_embed(const void* X, int64_t N, int d, int dtype, const float* params, float* E,
                      void* ws, size_t ws_bytes, cudaStream_t st) {
    const int Kp = (d + emb::KB - 1) / emb::KB * emb::KB;
    const int64_t chunk = emb_chunk(d);
    Carver cv(ws, ws_bytes);
    unsigned int* amax = cv.take<unsigned int>(4);
    float* inv_s = cv.take<float>(4);
    __half* XB = cv.take<__half>((size_t)emb_rows_buf(N, d) * Kp);
    __half* WB = cv.take<__half>((size_t)ml::HID * Kp);
    if (!cv.ok) return fail(ANN_ERR_WORKSPACE, "learned embed: workspace too small");
    if (N == 0) return ANN_OK;
    int rc = launch_absmax(X, dtype, N * d, nullptr, 0, amax, st);
    if (rc) return rc;
    k_inv_scale<<<1, 32, 0, st>>>(amax, inv_s);
    ANN_CHECK_LAUNCH();
    const float* W1 = params;
    const float* b1 = W1 + (int64_t)ml::HID * d;
    const float* W2 = b1 + ml::HID;
    const float* b2 = W2 + (int64_t)ml::OUT * ml::HID;
    k_to_half_rows<<<(unsigned)(((int64_t)ml::HID * Kp + 255) / 256), 256, 0, st>>>(
        W1, ANN_F32, d, 0, ml::HID, ml::HID, Kp, nullptr, WB);
    ANN_CHECK_LAUNCH();
    CUtensorMap tw;
    if ((rc = make_tmap(&tw, WB, ml::HID, Kp, emb::KB, ml::HID, CU_TENSOR_MAP_SWIZZLE_128B)))
        return rc;
    ANN_CHECK_CUDA(cudaFuncSetAttribute(k_embed_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)emb::SMEM));
    const uint32_t idesc = idesc_f16(emb::BM, ml::HID, 0);  // FP16 x FP16 -> FP32
    int* status = device_status_ptr();
    for (int64_t r0 = 0; r0 < N; r0 += chunk) {
        const int64_t n = N - r0 < chunk ? N - r0 : chunk;
        const int64_t n_pad = (n + emb::BM - 1) / emb::BM * emb::BM;  // <= emb_rows_buf
        const int64_t tot = n_pad * Kp;
        const unsigned g = (unsigned)((tot + 255) / 256 < 152 * 64 ? (tot + 255) / 256 : 152 * 64);
        k_to_half_rows<<<g, 256, 0, st>>>(X, dtype, d, r0, n, n_pad, Kp, inv_s, XB);
        ANN_CHECK_LAUNCH();
        CUtensorMap tx;
        if ((rc = make_tmap(&tx, XB, n_pad, Kp, emb::KB, emb::BM, CU_TENSOR_MAP_SWIZZLE_128B)))
            return rc;
        k_embed_tc<<<(unsigned)((n + emb::BM - 1) / emb::BM), emb::THREADS, emb::SMEM, st>>>(
            tx, tw, n, Kp / emb::KB, idesc, b1, W2, b2, E + r0 * ml::OUT, status);
        ANN_CHECK_LAUNCH();
    }
    return ANN_OK;
}

// ---- training ----------------------------------------------------------------
static constexpr int EST_K = 64;  // embedding-space list width of the recall estimate

struct LearnTrainWs {
    uint8_t* Q;          // [S x d] sample rows, X's type
    uint32_t* kq_id;     // [S x (kk+1)]
    float* kq_d;
    uint32_t* knn;       // [S x kk]
    void* qws;           // query workspace (exact, original space; then embedding space)
    size_t qws_bytes;
    uint32_t* idx;       // [3B]
    float *U, *H, *Z, *dZ, *dU;
    float *G, *m, *v;    // [P]
    float* li;           // [B]
    float* E;            // [N x 32]
    float* QE;           // [S x 32]
    uint32_t* eid;       // [S x EST_K]
    float* ed;
    unsigned long long* hits;
    int* step;           // device step counter (read by the captured step)
    float* part;         // split-K partial products
    void* ews;           // embedding workspace
    size_t ews_bytes;
    __nv_bfloat16 *xb, *xbt, *w1b, *dut;  // BF16 operands of the layer-1 GEMMs
};

// The sample's neighbour lists: the exact plan when it fits shared memory, else
// (FP32 at large d) scaled-FP16 screening of 128 candidates with the FP32 re-rank.
static int sample_plan(int d, int dtype, int kq, KnnPlan* p) {
    if (knn_plan(d, dtype, kq, ANN_EXACT, 0, p) == ANN_OK) return ANN_OK;
    return knn_plan(d, dtype, kq, ANN_F16_RERANK, 0, p);
}

// Buffers of one batch of B triplets (R = 3B rows, Rp = R rounded up to 128,
// Kp = d rounded up to 64): FP32 activations and gradients, and the split BF16
// operands of the tensor-core layer-1 GEMMs.
struct BatchBufs {
    float *U, *H, *Z, *dZ, *dU, *li, *part;
    __nv_bfloat16 *xb, *xbt, *w1b, *dut;  // [Rp x 3Kp], [Kp x 3Rp], [256 x 3Kp], [256 x 3Rp]
};
static inline int64_t batch_rp(int64_t B) { return (3 * B + 127) / 128 * 128; }
static inline int batch_kp(int d) { return (d + 63) / 64 * 64; }
static void take_bf16(Carver& cv, int64_t B, int d, BatchBufs& b) {
    const int64_t Rp = batch_rp(B), Kp = batch_kp(d);
    b.xb = cv.take<__nv_bfloat16>((size_t)(Rp * 3 * Kp));
    b.xbt = cv.take<__nv_bfloat16>((size_t)(Kp * 3 * Rp));
    b.w1b = cv.take<__nv_bfloat16>((size_t)(ml::HID * 3 * Kp));
    b.dut = cv.take<__nv_bfloat16>((size_t)(ml::HID * 3 * Rp));
}

// Loss and gradient of one batch: rows idx[0, B) anchors, [B, 2B) positives,
// [2B, 3B) negatives; G = [dW1 | db1 | dW2 | db2] (the layout of params); the
// mean loss into losses[*step] when losses is not NULL.
static int batch_grads(const void* X, int dtype, int d, const uint32_t* idx, int B,
                       const float* params, const float* inv_s, float margin, const BatchBufs& b,
                       float* G, float* losses, const int* step, cudaStream_t q) {
    const int64_t R = 3 * (int64_t)B, Rp = batch_rp(B);
    const int Kp = batch_kp(d);
    const float* W1 = params;
    const float* b1 = W1 + (int64_t)ml::HID * d;
    const float* b2 = b1 + ml::HID + (int64_t)ml::OUT * ml::HID;
    float* gW1 = G;
    float* gb1 = gW1 + (int64_t)ml::HID * d;
    float* gW2 = gb1 + ml::HID;
    float* gb2 = gW2 + (int64_t)ml::OUT * ml::HID;
    const float* W2 = params + (int64_t)ml::HID * d + ml::HID;
    int r;
    // layer 1 on the tensor cores: x / s and W1 split into BF16 parts (three
    // products), FP32 accumulation
    auto nb = [](int64_t n) { return (unsigned)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16); };
    k_batch_bf16<<<nb(Rp * Kp), 256, 0, q>>>(X, dtype, d, idx, R, Rp, Kp, inv_s, b.xb, b.xbt);
    ANN_CHECK_LAUNCH();
    k_w1_bf16<<<nb((int64_t)ml::HID * Kp), 256, 0, q>>>(W1, d, Kp, b.w1b);
    ANN_CHECK_LAUNCH();
    if ((r = gemm_tc(b.xb, Rp, b.w1b, ml::HID, 3 * Kp, R, ml::HID, 1,
                     EpTcHidden{b.U, b.H, b1, ml::HID}, q)))
        return r;
    // layer 2 in FP32
    if ((r = gemm(R, ml::OUT, ml::HID, mat(b.H, ANN_F32, ml::HID), mat(W2, ANN_F32, ml::HID, 1),
                  EpBias{b.Z, b2, ml::OUT}, q, b.part)))
        return r;
    k_triplet_loss<<<(B + 127) / 128, 128, 0, q>>>(b.Z, B, margin, b.dZ, b.li);
    ANN_CHECK_LAUNCH();
    if (losses) {
        k_mean<<<1, 256, 0, q>>>(b.li, B, step, losses);
        ANN_CHECK_LAUNCH();
    }
    // dW2 = dZ^T H, db2 = column sums of dZ
    if ((r = gemm(ml::OUT, ml::HID, (int)R, mat(b.dZ, ANN_F32, ml::OUT, 1),
                  mat(b.H, ANN_F32, ml::HID), EpStore{gW2, ml::HID}, q, b.part)))
        return r;
    k_colsum<<<1, 32, 0, q>>>(b.dZ, R, ml::OUT, gb2);
    ANN_CHECK_LAUNCH();
    // dU = (dZ W2) where U > 0
    if ((r = gemm(R, ml::HID, ml::OUT, mat(b.dZ, ANN_F32, ml::OUT), mat(W2, ANN_F32, ml::HID),
                  EpReluMask{b.dU, b.U, ml::HID}, q)))
        return r;
    // dW1 = dU^T (X / s) on the tensor cores (split BF16 operands, K = three
    // times the batch rows, split over K and summed in slice order), db1 =
    // column sums of dU
    k_du_bf16_t<<<nb((int64_t)ml::HID * Rp), 256, 0, q>>>(b.dU, R, Rp, b.dut);
    ANN_CHECK_LAUNCH();
    {
        const int nkb = (int)(3 * Rp / tgm::KB);
        int nz = nkb < 8 ? nkb : 8;
        while (nz > 1 && (int64_t)nz * ml::HID * d > SPLIT_PART_FLOATS) --nz;
        const int per = (nkb + nz - 1) / nz;
        nz = (nkb + per - 1) / per;
        if ((r = gemm_tc(b.dut, ml::HID, b.xbt, Kp, (int)(3 * Rp), ml::HID, d, nz,
                         EpTcPart{b.part, ml::HID, d}, q)))
            return r;
        k_split_reduce<<<(unsigned)(((int64_t)ml::HID * d + 255) / 256), 256, 0, q>>>(
            b.part, nz, ml::HID, d, EpStore{gW1, d});
        ANN_CHECK_LAUNCH();
    }
    k_colsum<<<1, 256, 0, q>>>(b.dU, R, ml::HID, gb1);
    ANN_CHECK_LAUNCH();
    return ANN_OK;
}

static size_t learned_grad_ws(int64_t B, int d, float** bufs_out, BatchBufs* bb_out, void* base,
                              size_t cap) {
    Carver cv(base, cap);
    const int64_t R = 3 * B;
    float* p[10];
    p[0] = cv.take<float>((size_t)R * ml::HID);   // U
    p[1] = cv.take<float>((size_t)R * ml::HID);   // H
    p[2] = cv.take<float>((size_t)R * ml::OUT);   // Z
    p[3] = cv.take<float>((size_t)R * ml::OUT);   // dZ
    p[4] = cv.take<float>((size_t)R * ml::HID);   // dU
    p[5] = cv.take<float>((size_t)B);             // li
    p[6] = cv.take<float>((size_t)SPLIT_PART_FLOATS);
    p[7] = cv.take<float>(4);                     // amax bits, inverse scale
    p[8] = cv.take<float>(4);                     // step (zero)
    p[9] = (float*)cv.take<uint32_t>((size_t)R);  // the batch's row ids, checked
    if (bufs_out)
        for (int i = 0; i < 10; ++i) bufs_out[i] = p[i];
    if (bb_out) {
        take_bf16(cv, B, d, *bb_out);
    } else {
        BatchBufs tmp;
        take_bf16(cv, B, d, tmp);
    }
    return cv.used + 256;
}

__global__ void k_checked_rows(const uint32_t* __restrict__ rows, int64_t n, int64_t N,
                               uint32_t* __restrict__ out, int* status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = safe_id(rows[i], N, status);
}

size_t learned_grad_bytes(int64_t B, int d) {
    return learned_grad_ws(B, d, nullptr, nullptr, nullptr, 0);
}

int run_learned_grad(const void* X, int64_t N, int d, int dtype, const float* params,
                     const uint32_t* rows, int B, float margin, float* grads, float* loss,
                     void* ws, size_t ws_bytes, cudaStream_t st) {
    float* p[10];
    BatchBufs bb;
    if (learned_grad_ws(B, d, p, &bb, ws, ws_bytes) > ws_bytes)
        return fail(ANN_ERR_WORKSPACE, "learned grad: workspace too small");
    unsigned int* amax = (unsigned int*)p[7];
    float* inv_s = p[7] + 1;
    int* step = (int*)p[8];
    uint32_t* idx = (uint32_t*)p[9];
    int rc;
    k_checked_rows<<<(unsigned)((3 * (int64_t)B + 255) / 256), 256, 0, st>>>(
        rows, 3 * (int64_t)B, N, idx, device_status_ptr());
    ANN_CHECK_LAUNCH();
    if ((rc = launch_absmax(X, dtype, N * d, nullptr, 0, amax, st))) return rc;
    k_inv_scale<<<1, 32, 0, st>>>(amax, inv_s);
    ANN_CHECK_LAUNCH();
    ANN_CHECK_CUDA(cudaMemsetAsync(step, 0, sizeof(int), st));
    bb.U = p[0];
    bb.H = p[1];
    bb.Z = p[2];
    bb.dZ = p[3];
    bb.dU = p[4];
    bb.li = p[5];
    bb.part = p[6];
    return batch_grads(X, dtype, d, idx, B, params, inv_s, margin, bb, grads, loss, step, st);
}

size_t learned_train_ws(int64_t N, int d, int dtype, int64_t S, int kk, int batch,
                        LearnTrainWs* out, void* base, size_t cap) {
    KnnPlan p1, p2;
    if (sample_plan(d, dtype, kk + 1, &p1) || knn_plan(ml::OUT, ANN_F32, EST_K, ANN_EXACT, 0, &p2))
        return 0;
    const size_t q1 = query_ws(N, S, p1, nullptr, nullptr, 0);
    const size_t q2 = query_ws(N, S, p2, nullptr, nullptr, 0);
    Carver cv(base, cap);
    LearnTrainWs w;
    const int64_t R = 3 * (int64_t)batch;
    const int64_t P = ml::n_params(d);
    w.Q = cv.take<uint8_t>((size_t)S * d * dtype_bytes(dtype));
    w.kq_id = cv.take<uint32_t>((size_t)S * (kk + 1));
    w.kq_d = cv.take<float>((size_t)S * (kk + 1));
    w.knn = cv.take<uint32_t>((size_t)S * kk);
    w.qws_bytes = q1 > q2 ? q1 : q2;
    w.qws = cv.take<uint8_t>(w.qws_bytes);
    w.idx = cv.take<uint32_t>((size_t)R);
    w.U = cv.take<float>((size_t)R * ml::HID);
    w.H = cv.take<float>((size_t)R * ml::HID);
    w.Z = cv.take<float>((size_t)R * ml::OUT);
    w.dZ = cv.take<float>((size_t)R * ml::OUT);
    w.dU = cv.take<float>((size_t)R * ml::HID);
    w.G = cv.take<float>((size_t)P);
    w.m = cv.take<float>((size_t)P);
    w.v = cv.take<float>((size_t)P);
    w.li = cv.take<float>((size_t)batch);
    w.E = cv.take<float>((size_t)N * ml::OUT);
    w.QE = cv.take<float>((size_t)S * ml::OUT);
    w.eid = cv.take<uint32_t>((size_t)S * EST_K);
    w.ed = cv.take<float>((size_t)S * EST_K);
    w.hits = cv.take<unsigned long long>(1);
    w.step = cv.take<int>(4);
    w.part = cv.take<float>((size_t)SPLIT_PART_FLOATS);
    w.ews_bytes = learned_embed_ws(N, d);
    w.ews = cv.take<uint8_t>(w.ews_bytes);
    BatchBufs bb;
    take_bf16(cv, batch, d, bb);
    w.xb = bb.xb;
    w.xbt = bb.xbt;
    w.w1b = bb.w1b;
    w.dut = bb.dut;
    if (out) *out = w;
    if (!base) return cv.used + 256;  // size query
    return cv.ok ? cv.used + 256 : 0;
}

int run_learned_train(const void* X, int64_t N, int d, int dtype, const uint32_t* sample,
                      int64_t S, int kk, int kpos, const uint32_t* draws, int steps, int batch,
                      float lr, float margin, float* params, float* losses, float* recall_est,
                      void* ws, size_t ws_bytes, cudaStream_t st) {
    LearnTrainWs w;
    const size_t need = learned_train_ws(N, d, dtype, S, kk, batch, &w, ws, ws_bytes);
    if (!need || need > ws_bytes) return fail(ANN_ERR_WORKSPACE, "learned train: workspace too small");
    int rc;
    const int64_t P = ml::n_params(d);
    const int64_t R = 3 * (int64_t)batch;
    // 1. exact kk nearest vectors of every sampled row (tile query kernel, all N)
    const int64_t rb = (int64_t)d * dtype_bytes(dtype);
    int* status = device_status_ptr();
    k_gather_rows<<<(unsigned)((S * 32 + 255) / 256), 256, 0, st>>>((const uint8_t*)X, rb, sample,
                                                                   S, N, w.Q, status);
    ANN_CHECK_LAUNCH();
    KnnPlan p1;
    if ((rc = sample_plan(d, dtype, kk + 1, &p1))) return rc;
    QueryWs q1;
    query_ws(N, S, p1, &q1, w.qws, w.qws_bytes);
    if ((rc = run_knn_query(X, N, w.Q, S, d, dtype, kk + 1, p1, q1, w.kq_id, w.kq_d, st)))
        return rc;
    k_drop_self<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(w.kq_id, kk + 1, sample, S, w.knn);
    ANN_CHECK_LAUNCH();
    // 2. input scale
    Carver ec(w.ews, w.ews_bytes);
    unsigned int* amax = ec.take<unsigned int>(4);
    float* inv_s = ec.take<float>(4);
    if ((rc = launch_absmax(X, dtype, N * d, nullptr, 0, amax, st))) return rc;
    k_inv_scale<<<1, 32, 0, st>>>(amax, inv_s);
    ANN_CHECK_LAUNCH();
    // 3. Adam steps
    ANN_CHECK_CUDA(cudaMemsetAsync(w.m, 0, (size_t)P * sizeof(float), st));
    ANN_CHECK_CUDA(cudaMemsetAsync(w.v, 0, (size_t)P * sizeof(float), st));
    // One training step; every step-dependent value is read from w.step on the
    // device, so the step can be captured once as a CUDA graph and replayed.
    auto one_step = [&](cudaStream_t q) -> int {
        int r;
        k_triplets<<<(batch + 255) / 256, 256, 0, q>>>(sample, S, w.knn, kk, kpos, draws,
                                                       w.step, batch, N, w.idx, status);
        ANN_CHECK_LAUNCH();
        BatchBufs bb{w.U, w.H, w.Z, w.dZ, w.dU, w.li, w.part, w.xb, w.xbt, w.w1b, w.dut};
        if ((r = batch_grads(X, dtype, d, w.idx, batch, params, inv_s, margin, bb, w.G,
                             losses, w.step, q)))
            return r;
        k_adam<<<(unsigned)((P + 255) / 256), 256, 0, q>>>(params, w.G, w.m, w.v, P, lr,
                                                           w.step);
        ANN_CHECK_LAUNCH();
        k_step_advance<<<1, 32, 0, q>>>(w.step);
        ANN_CHECK_LAUNCH();
        return ANN_OK;
    };
    ANN_CHECK_CUDA(cudaMemsetAsync(w.step, 0, sizeof(int), st));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    ANN_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
    if (steps > 1 && cs == cudaStreamCaptureStatusNone) {
        // Capture on a private stream ordered after st (the legacy default stream
        // cannot be captured), replay there, and order st after the replays.
        cudaStream_t q = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ANN_CHECK_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
        ANN_CHECK_CUDA(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
        ANN_CHECK_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
        ANN_CHECK_CUDA(cudaEventRecord(e0, st));
        ANN_CHECK_CUDA(cudaStreamWaitEvent(q, e0, 0));
        const unsigned long long l0 = ann_launch_count();  // counts the captured launches
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t ec = cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal);
        if (ec == cudaSuccess) {
            rc = one_step(q);
            ec = cudaStreamEndCapture(q, &g);
        }
        const unsigned long long per_step = ann_launch_count() - l0;
        if (!rc && ec == cudaSuccess) ec = cudaGraphInstantiate(&ge, g, 0);
        for (int t = 0; !rc && ec == cudaSuccess && t < steps; ++t) ec = cudaGraphLaunch(ge, q);
        if (!rc && ec == cudaSuccess) ec = cudaEventRecord(e1, q);
        if (!rc && ec == cudaSuccess) ec = cudaStreamWaitEvent(st, e1, 0);
        if (ge) cudaGraphExecDestroy(ge);  // freed once the queued launches finish
        if (g) cudaGraphDestroy(g);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(q);  // released once its work completes
        if (rc) return rc;
        if (ec != cudaSuccess)
            return fail(ANN_ERR_CUDA, "training step graph: %s", cudaGetErrorString(ec));
        count_launches(per_step * (unsigned long long)(steps - 1));
    } else {
        for (int t = 0; t < steps; ++t)
            if ((rc = one_step(st))) return rc;
    }
    // 4. recall estimate: the sample's exact top 10 within its top EST_K in
    //    embedding space (all N)
    if (recall_est) {
        if ((rc = run_learned_embed(X, N, d, dtype, params, w.E, w.ews, w.ews_bytes, st)))
            return rc;
        k_gather_rows<<<(unsigned)((S * 32 + 255) / 256), 256, 0, st>>>(
            (const uint8_t*)w.E, ml::OUT * 4, sample, S, N, (uint8_t*)w.QE, status);
        ANN_CHECK_LAUNCH();
        KnnPlan p2;
        if ((rc = knn_plan(ml::OUT, ANN_F32, EST_K, ANN_EXACT, 0, &p2))) return rc;
        QueryWs q2;
        query_ws(N, S, p2, &q2, w.qws, w.qws_bytes);
        if ((rc = run_knn_query(w.E, N, w.QE, S, ml::OUT, ANN_F32, EST_K, p2, q2, w.eid, w.ed, st)))
            return rc;
        ANN_CHECK_CUDA(cudaMemsetAsync(w.hits, 0, sizeof(unsigned long long), st));
        const int tk = kk < 10 ? kk : 10;
        k_cover<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(w.eid, EST_K, EST_K, w.knn, kk, tk,
                                                            S, w.hits);
        ANN_CHECK_LAUNCH();
        k_hits_to_recall<<<1, 32, 0, st>>>(w.hits, S * tk, recall_est);
        ANN_CHECK_LAUNCH();
    }
    return ANN_OK;
}

}  // namespace ann
