// Shared helpers of the sm_103a library: error state, launch checks, and thin
// inline-PTX wrappers for mbarrier, TMA (cp.async.bulk.tensor) and tcgen05.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/ann.h"

namespace ann {

// ---- host-side error state -------------------------------------------------
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);

#define ANN_CHECK_CUDA(expr)                                                       \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return ::ann::fail(ANN_ERR_CUDA, "%s: %s (%s:%d)", #expr,              \
                               cudaGetErrorString(e_), __FILE__, __LINE__);        \
    } while (0)

// Every kernel launch of the library is followed by ANN_CHECK_LAUNCH(), which
// also counts it (ann_launch_count).
void count_launch();
void count_launches(unsigned long long n);  // kernels run by graph replays
#define ANN_CHECK_LAUNCH()                \
    do {                                  \
        ::ann::count_launch();            \
        ANN_CHECK_CUDA(cudaGetLastError()); \
    } while (0)

// Optional CUDA-event timing of the distance-tile kernel (ann_timing_enable).
struct TileTimer {
    cudaEvent_t a = nullptr, b = nullptr;
};
bool tile_timing_on();
void tile_timing_record(cudaEvent_t a, cudaEvent_t b);
cudaEvent_t tile_event();
// Optional cycle/event counters inside the distance-tile kernel (ann_tile_counters_*).
bool tile_counters_on();
int tile_counters_read(unsigned long long* out, int n, bool reset);

#define ANN_REQUIRE(cond, ...)                                                     \
    do {                                                                           \
        if (!(cond)) return ::ann::fail(ANN_ERR_INVALID_ARG, __VA_ARGS__);         \
    } while (0)

// ---- device-side status word (timeouts, violated preconditions) -----------
// Bits: ANN_DEV_TIMEOUT, ANN_DEV_BAD_INPUT, ANN_DEV_OVERFLOW.  Read and cleared
// by ann_device_status().
enum : int { DEV_TIMEOUT = 1, DEV_BAD_INPUT = 2, DEV_OVERFLOW = 4 };
int* device_status_ptr();  // device address of the status word (current device)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Sub-allocator over a caller workspace.  Each carve is 256-byte aligned.
struct Carver {
    char* base;
    size_t cap, used = 0;
    bool ok = true;
    Carver(void* b, size_t c) : base((char*)b), cap(c) {}
    template <class T> T* take(size_t n) {
        size_t off = align_up(used, 256);
        used = off + n * sizeof(T);
        if (used > cap) ok = false;
        return (base && ok) ? (T*)(base + off) : nullptr;
    }
};

inline int dtype_bytes(int dt) { return dt == ANN_U8 ? 1 : (dt == ANN_F32 ? 4 : 2); }

// ---- device helpers ---------------------------------------------------------
__device__ __forceinline__ float load_elem(const void* X, int dtype, int64_t i) {
    switch (dtype) {
    case ANN_F32: return __ldg((const float*)X + i);
    case ANN_F16: return __half2float(__ldg((const __half*)X + i));
    case ANN_BF16: return __bfloat162float(__ldg((const __nv_bfloat16*)X + i));
    default: return (float)__ldg((const uint8_t*)X + i);
    }
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Order-preserving map of a float onto uint32 (for composite (key, index) sorts).
__device__ __forceinline__ uint32_t f2ord(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier -----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete, giving up after
// limit_ns of wall time or as soon as *abort is set.  Returns false when it
// gave up; the caller must then stop its loop.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0) {
            if (*abort) return false;
            if (globaltimer() - t0 > limit_ns) {
                *abort = 1;
                return false;
            }
        }
    }
}

// ---- 32-bit shared-memory accesses by address ------------------------------------
__device__ __forceinline__ void sts_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// ---- TMA ----------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// ---- tcgen05 --------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (FP16 or BF16 inputs, FP32 accumulator).
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive once on the mbarrier when every tcgen05.mma issued so far by this thread completes.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread t gets lane (taddr.lane + t).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle (8-row x 128-byte atoms, atoms 1024 bytes apart).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                     // layout: SWIZZLE_128B
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B of one type
// (0 = FP16, 1 = BF16), both K-major, tile M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, uint32_t ab_fmt) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

}  // namespace ann
