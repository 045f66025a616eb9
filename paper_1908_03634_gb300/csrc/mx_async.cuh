// Per-thread asynchronous global -> shared copies (cp.async, sm_80 and later):
// element copies with zero fill, commit groups and waits on them.
#pragma once

// sizeof(T)-byte global -> shared copy of the first n bytes, the rest zero
// filled (n = 0: src names a valid address but no byte is read)
template <typename T>
__device__ __forceinline__ void cp_async_el(T *dst, const T *src, int n) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's most recent groups are in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// 16-byte global -> shared copy (both addresses 16-byte aligned) of the first n
// bytes (0 or 16), the rest zero filled; cached in L2 only
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int n) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
