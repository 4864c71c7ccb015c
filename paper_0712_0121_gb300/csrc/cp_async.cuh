// Asynchronous global -> shared copies (cp.async, no register round trip).
// The copies a thread issued complete at cp_async_wait<n> (all but its n
// most recent committed groups) and become visible to the CTA after a
// barrier.
#pragma once

#include <cstdint>

namespace morph {

__device__ __forceinline__ void cp_async4(uint32_t *sdst, const uint32_t *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
// both addresses 8-byte aligned
__device__ __forceinline__ void cp_async8(uint32_t *sdst, const uint32_t *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gsrc) : "memory");
}
// both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(uint32_t *sdst, const uint32_t *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace morph
