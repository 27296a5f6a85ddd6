// Per-thread asynchronous copies (global -> shared, cp.async) with zero fill:
// the staging primitive of the tiled stencil. Completion is awaited with
// cp.async.wait_group, which always returns once the thread's own copies
// have landed (no spinning on other threads).
#pragma once

#include <cstdint>

namespace fmp {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 8-byte cp.async with zero fill when !valid (src is not dereferenced then).
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
    const unsigned n = valid ? 8u : 0u;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace fmp
