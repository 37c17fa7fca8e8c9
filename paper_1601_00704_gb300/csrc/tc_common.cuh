// tc_common.cuh -- shared by the tensor-core (tcgen05, sm_103a) kernels of the
// warm-start network: nn_tc.cu (convolution forward, inference) and
// nn_tc_train.cu (training: weight gradients).  Inline-PTX wrappers for
// mbarriers, TMA tensor loads and tcgen05 (TMEM allocation, MMA, commit,
// loads), the shared-memory matrix descriptors, and host helpers.

#pragma once

#include "glbm.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

extern __attribute__((visibility("hidden"))) thread_local char g_create_err[512];

// defined in nn_tc.cu, library-internal: the debug-starve test hook and the
// kernel choice of glbm_nn_tc_set_variant
extern int g_tc_starve;
extern int g_tc_variant;

namespace {

constexpr int TC_M = 128;        // output pixels per tile (UMMA M)
constexpr int TC_KC = 32;        // input channels per K step: 64-byte rows
constexpr int TC_STAGES = 3;     // TMA ring depth (2, 3, 4 and 7-8 measured: 3 best, occupancy wins)
constexpr int TC_STAGES_DEEP = 8; // ring depth of grids with at most one CTA per SM
constexpr int TC_THREADS = 192;  // warp 0 TMA, warp 1 MMA + TMEM, warps 2-5 epilogue
constexpr int TC_STAGE_A = TC_M * TC_KC * 2;          // 8 KB
constexpr long long kWaitCycles = 4ll << 30;          // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// As mbar_try_wait, but a thread whose phase is not yet complete may sleep
// inside the instruction for up to `ns` nanoseconds (it wakes when the phase
// completes), so that waiting warps leave their scheduler's issue slots to
// the warps that work.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity.  Returns false (without
// waiting further) once any thread of the CTA has given up.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err, int code) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            atomicExch(err, code);
            return false;
        }
    }
    return true;
}
// mbar_wait for warps that only wait (the same bound, sleeping between tests).
__device__ bool mbar_wait_idle(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err, int code) {
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(bar, parity, 20000u)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            atomicExch(err, code);
            return false;
        }
    }
    return true;
}

// Teardown: wait, bounded and whatever the abort flag says, for a phase
// that work already in flight completes (TMA copies landing in shared memory,
// MMAs retiring), so that none of it outlives the CTA's shared or tensor
// memory after a timeout.  In a run without a timeout the phase has long
// completed and the test passes at once.
__device__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}
// The copies of the last min(S, issued) stage loads of an S-stage ring (no
// later load went into those stages, so their phases are the latest).
__device__ void drain_ring(uint64_t *full, int S, long long issued) {
    for (long long u = issued > S ? issued - S : 0; u < issued; ++u) mbar_drain(&full[u % S], uint32_t(u / S) & 1u);
}

// Test hook (glbm_nn_tc_debug_starve): stage number + 1 whose copies the
// first CTA of the next tensor-core launch leaves unissued, 0 for none.
inline int take_starve() {
    const int s = g_tc_starve;
    g_tc_starve = 0;
    return s;
}

// ---- TMA --------------------------------------------------------------------
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Shared -> global tensor copy in the CTA's bulk group; the threads that
// wrote the source must have made it visible to the async proxy
// (fence.proxy.async.shared::cta) before this thread issues the copy.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// until at most one committed group may still be reading its shared source
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// until no committed group is still reading its shared source
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// until every committed group has completed its writes
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---- tcgen05 ----------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulator.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The mbarrier receives one arrival when every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory matrix descriptor of a K-major tile whose rows are 64 bytes
// (32 BF16) with the 64-byte swizzle, as TMA writes it: 8-row groups 512 B
// apart (stride byte offset); the leading byte offset is unused for swizzled
// K-major tiles; bits 46-47 hold the descriptor version 1; bits 61-63 the
// swizzle mode (4 = 64 bytes).
__device__ __forceinline__ uint64_t sdesc_k64(const void *tile) {
    const uint64_t a = smem_u32(tile);
    return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((512ull >> 4) << 32) | (1ull << 46) | (4ull << 61);
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N/8 in bits
// 17-22, M/16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(TC_M >> 4) << 24);
}

int grid_for(long long total) {
    long long b = (total + 255) / 256;
    return int(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

glbm_status tcfail(glbm_status s, const char *msg) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
    return s;
}
glbm_status tccuda(cudaError_t e, const char *what) {
    snprintf(g_create_err, sizeof(g_create_err), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GLBM_ENOMEM : GLBM_ECUDA;
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

}  // namespace
