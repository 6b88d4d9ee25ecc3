// grid_common.cuh -- grid-wide helpers of the persistent (cooperative) kernels.
#pragma once

#include "device_common.cuh"

namespace snn {

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t x;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(x) : "l"(p) : "memory");
    return x;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Split barrier: grid_arrive publishes this CTA's arrival (after all its
// threads' earlier writes), grid_wait waits for `expected` arrivals of the
// current barrier.  Between the two a CTA may only do work that reads nothing
// another CTA wrote before the barrier.  `gen` counts this CTA's barriers
// (thread 0's copy is the one used).
__device__ inline void grid_arrive(DevState* st, uint32_t& gen) {
    __syncthreads();
    if (threadIdx.x == 0) {
        gen += 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&st->bar_count) : "memory");
    }
}

__device__ inline bool grid_wait(DevState* st, uint32_t expected, uint64_t limit_ns, uint32_t gen) {
    __shared__ int s_okw;
    if (threadIdx.x == 0) {
        const uint32_t target = expected * gen;
        int ok = 1;
        if ((int32_t)(ld_acquire(&st->bar_count) - target) < 0) {
            const uint64_t start = global_ns();
            while ((int32_t)(ld_acquire(&st->bar_count) - target) < 0) {
                if (global_ns() - start > limit_ns) {
                    atomicOr(&st->err, ERR_BARRIER_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ok && ld_acquire(&st->err) != 0) ok = 0;
        s_okw = ok;
    }
    __syncthreads();
    return s_okw != 0;
}

// Barrier over `expected` CTAs on the arrival counter of `st` (all CTAs are
// co-resident: cooperative launch).  The counter starts at 0 for every launch
// (the host clears it) and only grows: the k-th barrier of the launch is
// passed once it reaches expected * k, so arriving is a single release
// reduction with no round trip and no reset.  `gen` counts this CTA's
// barriers (start it at 0).  Returns false if this CTA's wait ran out (after
// limit_ns of the global timer; it then sets ERR_BARRIER_TIMEOUT) or another
// CTA reported an error.
__device__ inline bool grid_barrier_on(DevState* st, uint32_t expected, uint64_t limit_ns, uint32_t& gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        gen += 1;
        const uint32_t target = expected * gen;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&st->bar_count) : "memory");
        int ok = 1;
        if ((int32_t)(ld_acquire(&st->bar_count) - target) < 0) {
            const uint64_t start = global_ns();
            while ((int32_t)(ld_acquire(&st->bar_count) - target) < 0) {
                if (global_ns() - start > limit_ns) {
                    atomicOr(&st->err, ERR_BARRIER_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ok && ld_acquire(&st->err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Barrier over the G CTAs that simulate network v.
__device__ inline bool grid_barrier(const NetView& v, uint32_t G, uint32_t& gen) {
    return grid_barrier_on(v.st, G + v.barrier_extra, v.wait_limit_ns, gen);
}

// Exclusive prefix of cnt[0..n) (global, written by other CTAs) into
// out[0..n] (shared), out[n] = total: coalesced loads, eight per thread in
// flight before the first is stored (one L2 round trip for n <= 8 x threads;
// a loop that stores each load before issuing the next pays one per pass),
// then the scan in shared memory.
__device__ inline void block_scan_inplace(uint32_t* s, uint32_t n);
__device__ inline void block_exclusive_scan(const uint32_t* cnt, uint32_t n, uint32_t* out) {
    for (uint32_t base = 0; base < n; base += 8 * blockDim.x) {
        uint32_t x[8];
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) {
            const uint32_t i = base + k * blockDim.x + threadIdx.x;
            x[k] = i < n ? __ldcg(cnt + i) : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) {
            const uint32_t i = base + k * blockDim.x + threadIdx.x;
            if (i < n) out[i] = x[k];
        }
    }
    __syncthreads();
    block_scan_inplace(out, n);
}

// Neuron id of staged spike j: CTA by binary search over the CTA offsets,
// warp by a scan of that CTA's W warp offsets, then the warp's segment.
template <int W>
__device__ __forceinline__ uint32_t spike_id(const NetView& v, const uint32_t* s_cta, const uint32_t* s_woff,
                                             uint32_t j, uint32_t Q, uint32_t TW, uint32_t G) {
    uint32_t lo = 0, hi = G;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_cta[mid] <= j)
            lo = mid;
        else
            hi = mid;
    }
    const uint32_t jl = j - s_cta[lo];
    uint32_t w = 0;
#pragma unroll
    for (uint32_t k = 1; k < (uint32_t)W; ++k)
        if (s_woff[lo * W + k] <= jl) w = k;
    const uint32_t wg = lo * W + w;
    const uint32_t qa = (uint32_t)((uint64_t)Q * wg / TW);
    return __ldcg(v.seg + ((size_t)qa << 2) + (jl - s_woff[wg]));
}

// In-place exclusive prefix of s[0..n) in shared memory, s[n] = total.
__device__ inline void block_scan_inplace(uint32_t* s, uint32_t n) {
    __shared__ uint32_t s_w2[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t a = min(threadIdx.x * per, n), b = min(a + per, n);
    uint32_t local = 0;
    for (uint32_t i = a; i < b; ++i) local += s[i];
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) s_w2[warp] = incl;
    __syncthreads();
    uint32_t base = 0, total = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
        if (w < warp) base += s_w2[w];
        total += s_w2[w];
    }
    uint32_t run = base + incl - local;
    for (uint32_t i = a; i < b; ++i) {
        const uint32_t x = s[i];
        s[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) s[n] = total;
    __syncthreads();
}

}  // namespace snn
