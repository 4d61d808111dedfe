// Small device helpers for the packed int16x2 kernels: byte permute, the
// selector that builds a packed profile addend from two residues' rows, the
// asynchronous 16-byte global -> shared copy and a broadcast of a 16-bit
// value to both halves.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace swdb {
namespace simd16 {

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Selector taking byte c of a (low half) and byte c of b (high half), each
// sign-extended to 16 bits.
__host__ __device__ constexpr uint32_t pair_sel(int c) {
    return uint32_t(c) | (uint32_t(c | 8) << 4) | (uint32_t(4 + c) << 8) | (uint32_t((4 + c) | 8) << 12);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// v (taken modulo 2^16) in both halves.
__host__ __device__ __forceinline__ uint32_t pack2(int v) {
    const uint32_t h = uint32_t(v) & 0xffffu;
    return h | (h << 16);
}

}  // namespace simd16
}  // namespace swdb
