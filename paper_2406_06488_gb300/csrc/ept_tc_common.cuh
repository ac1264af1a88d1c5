// ept_tc_common.cuh -- helpers shared by libept's tcgen05 kernels: mbarriers with
// bounded waits, TMA tile loads, tensor-memory fences and loads, shared-memory matrix
// descriptors and the 16-bit MMA (kind::f16 with FP16 operands, cta_group::1, FP32
// accumulation).
#pragma once
#include <cuda.h>
#include <cstdint>

#include "ept_internal.cuh"

namespace ept {
namespace tc {

// every mbarrier wait gives up after this long (then the kernel records an error
// code, raises its CTA abort flag, drains its own asynchronous work and returns)
constexpr unsigned long long WAIT_NS = 2000000000ull;   // default limit of a bounded wait (Batch::wait_ns)

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One test of a phase: the thread may sleep in the wait until the phase completes
// or TRY_WAIT_NS pass (then false), so that waiting warps leave the issue slots to
// the others.  Every 256 tests of mbar_wait below are then at most about 8 ms.
constexpr uint32_t TRY_WAIT_NS = 32768;
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(TRY_WAIT_NS)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed; false when the CTA is aborting or
// the wait expired (then the abort flag is raised and the error recorded).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          Counters *ctr, unsigned long long code, unsigned long long limit) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            const unsigned long long now = gtimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit) {
                *abort_flag = 1;
                atomicCAS(&ctr->err_code, 0ull, code);
                return false;
            }
        }
    }
}

// Bounded wait on a device word becoming non-zero (the same limit and abort
// protocol as mbar_wait).
__device__ __forceinline__ bool flag_wait(const volatile unsigned int *flag, volatile int *abort_flag, Counters *ctr,
                                          unsigned long long code, unsigned long long limit) {
    const unsigned long long t0 = gtimer();
    for (;;) {
        if (*flag) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > limit) {
            *abort_flag = 1;
            atomicCAS(&ctr->err_code, 0ull, code);
            return false;
        }
        __nanosleep(1000);
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void *tmap, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: start address >> 4
// (bits 0-13), leading byte offset 16 B (unused for swizzled K-major), stride byte
// offset 1024 B between 8-row groups (bits 32-45), descriptor version 1 (bit 46),
// swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Shared-memory matrix descriptor of a K-major tile in the 64-byte swizzle layout:
// rows of 64 bytes (32 16-bit values), 8-row atoms of 512 bytes (stride byte offset
// 512), the 16-byte chunks of row r XOR-swizzled by (r / 2) mod 4 (layout type 4).
// Stepping K by 16 elements inside the row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = FP16 (format 0
// in bits 7-9 and 10-12), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) += A (smem) * B (smem)^T, or D = A * B^T when accumulate == 0;
// issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 0/1 bits of `byte` -> eight FP16 values (1.0 = 0x3C00), element e = bit e.
__device__ __forceinline__ uint4 expand8(uint32_t byte) {
    uint4 v;
    v.x = (byte & 1u) * 0x3C00u + (byte & 2u) * 0x1E000000u;
    v.y = ((byte >> 2) & 1u) * 0x3C00u + ((byte >> 2) & 2u) * 0x1E000000u;
    v.z = ((byte >> 4) & 1u) * 0x3C00u + ((byte >> 4) & 2u) * 0x1E000000u;
    v.w = ((byte >> 6) & 1u) * 0x3C00u + ((byte >> 6) & 2u) * 0x1E000000u;
    return v;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tc
}  // namespace ept
