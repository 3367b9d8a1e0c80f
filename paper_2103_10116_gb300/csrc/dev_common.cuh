// dev_common.cuh -- device helpers: deterministic reductions, last-block
// detection, mbarrier + 1-D bulk (TMA) copies with bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spx_internal.cuh"

namespace spx {

// ------------------------------------------------------------------ reductions
// Fixed shuffle pattern => the same inputs always give the same bits.
template <class T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of v; the result is valid in every thread.  red must hold
// BLOCK/32 elements; the call ends with the buffer free for reuse.
__device__ __forceinline__ int warp_max(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <class T, int BLOCK> __device__ __forceinline__ T block_sum(T v, T *red)
{
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    constexpr int NW = BLOCK / 32;
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    T s = T(0);
    if (w == 0) {
        s = l < NW ? red[l] : T(0);
        s = warp_sum(s);
        if (l == 0) red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// Last-block detection (threadfence reduction pattern).  Every block calls
// it once, after its global writes; it returns true in exactly one block, the
// last to arrive, which then sees all other blocks' writes.  The last block
// resets the counter for the next launch in stream order.
__device__ __forceinline__ bool last_block(unsigned *ticket, unsigned nblocks)
{
    __shared__ unsigned s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(ticket, 1u);
        s_last = (prev == nblocks - 1) ? 1u : 0u;
        if (s_last) *ticket = 0u;
    }
    __syncthreads();
    const bool last = s_last != 0u;
    if (last) __threadfence();
    return last;
}

// L1-bypassing loads for data written by other blocks of the same launch.
template <class T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// ------------------------------------------------------------------ mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar`.  dst, src and
// bytes must be multiples of 16 (the callers round ranges outwards inside
// padded allocations).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Bounded wait for phase `parity` of `bar`: gives up after about `limit_cycles`
// SM clock cycles, sets DEVERR_MBAR_TIMEOUT in *err and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err,
                                          long long limit_cycles = 2000000000LL)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit_cycles) {
            if (err) atomicOr(err, DEVERR_MBAR_TIMEOUT);
            return false;
        }
    }
    return true;
}

}  // namespace spx
