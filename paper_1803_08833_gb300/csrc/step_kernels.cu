// step_kernels.cu -- one simulation time step (Sec. II-A, flow steps 1-6).
//
//   k_neuron_step  flow steps 1, 4-6 for every neuron: read and clear this step's
//                  delay-ring slot, add the external Poisson input, integrate
//                  Eq. 1-2 exactly over dt, threshold / reset / refractory /
//                  adaptation; the block's spikes are compacted in id order.
//                  The last block to finish turns the per-block spike counts
//                  into offsets, so spikes have a global (step, id) order
//                  without any inter-block waiting.
//   k_deliver      flow steps 2-4: every spike of the step adds its K weights,
//                  in int32 fixed point, into ring[(t + delay) mod D][target]
//                  with fire-and-forget L2 reductions; it also writes the
//                  (step, id) raster entries.
#include "device_common.cuh"

#include <cuda_bf16.h>

namespace snn {

// Last block of the neuron kernel: exclusive prefix of the per-block spike
// counts (block offsets) and the bookkeeping of the step.  Each warp scans a
// contiguous range of blocks in 32-wide coalesced chunks.
__device__ __forceinline__ void finish_step(const NetView& v, uint32_t t) {
    constexpr int W = NEURON_THREADS / 32;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nb = v.nb;
    const uint32_t range = (((nb + W - 1) / W) + 31) & ~31u;
    const uint32_t b0 = warp * range, b1 = min(b0 + range, nb);
    __shared__ uint32_t s_wtot[W];
    __shared__ unsigned long long s_wext[W], s_wrec[W];
    uint32_t tot = 0;
    unsigned long long ext = 0, rec = 0;
#pragma unroll 4
    for (uint32_t b = b0 + lane; b < b1; b += 32) {
        tot += __ldcg(v.blk_cnt + b);
        ext += __ldcg(reinterpret_cast<const unsigned long long*>(v.blk_ext) + b);
        if (v.row_len) rec += __ldcg(reinterpret_cast<const unsigned long long*>(v.blk_rec) + b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
        ext += __shfl_xor_sync(0xFFFFFFFFu, ext, o);
        rec += __shfl_xor_sync(0xFFFFFFFFu, rec, o);
    }
    if (lane == 0) {
        s_wtot[warp] = tot;
        s_wext[warp] = ext;
        s_wrec[warp] = rec;
    }
    __syncthreads();
    uint32_t base = 0, total = 0;
    unsigned long long ext_total = 0, rec_total = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        if (w < (int)warp) base += s_wtot[w];
        total += s_wtot[w];
        ext_total += s_wext[w];
        rec_total += s_wrec[w];
    }
    for (uint32_t c = b0; c < b1; c += 32) {
        const uint32_t b = c + lane;
        const uint32_t x = b < b1 ? __ldcg(v.blk_cnt + b) : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (b < b1) v.blk_off[b] = base + incl - x;
        base += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (threadIdx.x == 0) {
        DevState* st = v.st;
        v.blk_off[nb] = total;
        st->n_spk = total;
        st->t_deliver = t;
        st->raster_base = st->raster_count;
        st->raster_count += total;
        st->n_spikes += total;
        st->rec_events += v.row_len ? (uint64_t)rec_total : (uint64_t)total * v.K;
        st->ext_events += ext_total;
        st->t = t + 1;
        st->done = 0;
    }
}

__global__ void __launch_bounds__(NEURON_THREADS) k_neuron_step(NetView v) {
    __shared__ uint32_t s_t;
    __shared__ bool s_last;
    __shared__ uint32_t s_pois[MAX_POIS];
    if (threadIdx.x == 0) s_t = v.st->t;  // one read per block, not per thread
    load_poisson_table(v, s_pois);
    __syncthreads();
    const uint32_t t = s_t;
    const uint32_t slot = t % v.D;
    const uint32_t tid = threadIdx.x;
    const uint32_t base = blockIdx.x * NEURONS_PER_BLOCK + tid * NEURONS_PER_THREAD;

    uint32_t next_sum = 0;
    uint64_t rec = 0;
    const uint32_t spk = update_quad(v, s_pois, base, t, slot, next_sum, rec);

    // Block-ordered compaction: exclusive prefix of per-thread spike counts.
    const uint32_t lane = tid & 31, warp = tid >> 5;
    const uint32_t cnt = __popc(spk);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += x;
    }
    uint32_t ext_w = next_sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ext_w += __shfl_xor_sync(0xFFFFFFFFu, ext_w, o);
        rec += __shfl_xor_sync(0xFFFFFFFFu, rec, o);
    }
    __shared__ uint32_t s_wsum[NEURON_THREADS / 32];
    __shared__ uint32_t s_wext[NEURON_THREADS / 32];
    __shared__ unsigned long long s_wrec[NEURON_THREADS / 32];
    if (lane == 31) s_wsum[warp] = incl;
    if (lane == 0) {
        s_wext[warp] = ext_w;
        s_wrec[warp] = rec;
    }
    __syncthreads();
    uint32_t woff = 0, btot = 0, bext = 0;
    unsigned long long brec = 0;
#pragma unroll
    for (int w = 0; w < NEURON_THREADS / 32; ++w) {
        const uint32_t x = s_wsum[w];
        if (w < (int)warp) woff += x;
        btot += x;
        bext += s_wext[w];
        brec += s_wrec[w];
    }
    uint32_t pos = woff + incl - cnt;
    uint32_t* seg = v.seg + (size_t)blockIdx.x * NEURONS_PER_BLOCK;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (spk & (1u << q)) {
            if (SNN_BOUND(v.st, pos < (uint32_t)NEURONS_PER_BLOCK)) seg[pos] = base + q;
            ++pos;
        }

    if (tid == 0) {
        v.blk_cnt[blockIdx.x] = btot;
        v.blk_ext[blockIdx.x] = bext;
        if (v.row_len) v.blk_rec[blockIdx.x] = brec;
        __threadfence();
        const uint32_t ticket = atomicAdd(&v.st->done, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // All other blocks have published their counts (each fenced before its ticket).
    __threadfence();
    finish_step(v, t);
}

// ---------------------------------------------------------------------------
// Delivery.  The staged spikes of the step are addressed by their global
// index j; the owning neuron block is found by binary search over the block
// offsets (held in shared memory).

__device__ __forceinline__ uint32_t find_block(const uint32_t* s_off, uint32_t nb, uint32_t j) {
    // largest b with s_off[b] <= j (s_off[0] = 0, s_off[nb] = n_spk > j)
    uint32_t lo = 0, hi = nb;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_off[mid] <= j)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// AER raster (Sec. II-C): entry rbase + j = (step, id of staged spike j).
__device__ __forceinline__ void write_raster(const NetView& v, const uint32_t* s_off, uint32_t n_spk,
                                             uint32_t t, uint64_t rbase) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_spk; j += stride) {
        const uint64_t r = rbase + j;
        if (r >= v.raster_cap) break;
        const uint32_t b = find_block(s_off, v.nb, j);
        v.raster_t[r] = t;
        v.raster_id[r] = __ldcg(v.seg + (size_t)b * NEURONS_PER_BLOCK + (j - s_off[b]));
    }
}

// Per-launch header of the delivery kernels, read once per block.
struct StepHeader {
    uint32_t n_spk, t;
    uint64_t rbase;
};

__device__ __forceinline__ StepHeader read_header(const NetView& v) {
    __shared__ StepHeader s_h;
    if (threadIdx.x == 0) {
        s_h.n_spk = v.st->n_spk;
        s_h.t = v.st->t_deliver;
        s_h.rbase = v.st->raster_base;
    }
    __syncthreads();
    return s_h;
}

// Schedule 0: warps over (spike, 128-synapse chunk) tasks; each lane handles 4
// consecutive synapses (one 16 B target load, one 16 B f32 / 8 B bf16 weight
// load, one 4 B delay load).  The task range is split statically over the
// blocks (every chunk but a row's last has 128 synapses, so the split is even);
// a block first stages the ids of its spikes in shared memory, then each warp
// issues the loads of DELIVER_UNROLL tasks before their reductions, so several
// independent table reads are in flight per warp.
template <bool BF16>
__global__ void __launch_bounds__(256) k_deliver_warp(NetView v) {
    extern __shared__ uint32_t s_off[];  // nb + 1 block offsets, then blockDim.x staged ids
    const StepHeader h = read_header(v);
    if (h.n_spk == 0) return;
    const uint32_t nb = v.nb;
    for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) s_off[b] = v.blk_off[b];
    __syncthreads();
    write_raster(v, s_off, h.n_spk, h.t, h.rbase);

    const uint32_t chunks = (v.K + 127) >> 7;
    if (chunks == 0) return;
    const uint64_t n_tasks = (uint64_t)h.n_spk * chunks;
    const uint64_t t0 = n_tasks * blockIdx.x / gridDim.x;
    const uint64_t t1 = n_tasks * (blockIdx.x + 1) / gridDim.x;
    if (t0 >= t1) return;
    uint32_t* s_id = s_off + nb + 1;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t slot0 = h.t % v.D;
    const uint64_t pol = evict_first_policy();
    const uint32_t j_last = (uint32_t)((t1 - 1) / chunks);

    for (uint32_t jb = (uint32_t)(t0 / chunks); jb <= j_last; jb += blockDim.x) {
        const uint32_t j = jb + threadIdx.x;
        if (j <= j_last) {
            const uint32_t b = find_block(s_off, nb, j);
            s_id[threadIdx.x] = __ldcg(v.seg + (size_t)b * NEURONS_PER_BLOCK + (j - s_off[b]));
        }
        __syncthreads();
        const uint64_t lo = max(t0, (uint64_t)jb * chunks);
        const uint64_t hi = min(t1, (uint64_t)(jb + blockDim.x) * chunks);
        for (uint64_t tk = lo + warp; tk < hi; tk += (uint64_t)nwarps * DELIVER_UNROLL)
            deliver_tasks<BF16>(v, tk, nwarps, hi, chunks, s_id, jb, slot0, lane, pol);
        __syncthreads();
    }
}

// Schedule 1: one thread per synapse over the flattened (spike, synapse)
// range, scalar loads.
template <bool BF16>
__global__ void __launch_bounds__(256) k_deliver_thread(NetView v) {
    extern __shared__ uint32_t s_off[];
    const StepHeader h = read_header(v);
    if (h.n_spk == 0) return;
    const uint32_t nb = v.nb;
    for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) s_off[b] = v.blk_off[b];
    __syncthreads();
    write_raster(v, s_off, h.n_spk, h.t, h.rbase);
    const uint32_t slot0 = h.t % v.D;
    const uint64_t total = (uint64_t)h.n_spk * v.K;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t cached_j = 0xFFFFFFFFu, id = 0;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const uint32_t j = (uint32_t)(g / v.K);
        const uint32_t k = (uint32_t)(g - (uint64_t)j * v.K);
        if (j != cached_j) {
            const uint32_t b = find_block(s_off, nb, j);
            id = __ldcg(v.seg + (size_t)b * NEURONS_PER_BLOCK + (j - s_off[b]));
            cached_j = j;
        }
        if (v.row_len && k >= __ldg(v.row_len + id)) continue;  // past this row's end
        const size_t e = (size_t)id * v.Kpad + k;
        const uint32_t x = __ldg(v.td + e);
        const float w = BF16 ? __uint_as_float((uint32_t)__ldg(reinterpret_cast<const uint16_t*>(v.w) + e) << 16)
                             : __ldg(reinterpret_cast<const float*>(v.w) + e);
        uint32_t s = slot0 + (x >> 24);
        if (s >= v.D) s -= v.D;
        red_add(v.ring + (size_t)s * v.Npad + (x & 0xFFFFFFu), fx_weight(v, w));
    }
}

cudaError_t launch_neuron_step(const NetView& v, cudaStream_t s) {
    k_neuron_step<<<v.nb, NEURON_THREADS, 0, s>>>(v);
    count_launch(1);
    return cudaGetLastError();
}

// Dynamic shared memory of a delivery block: block offsets + staged spike ids.
static size_t deliver_smem(uint32_t nb, int block) { return (size_t)(nb + 1 + block) * sizeof(uint32_t); }

static const void* deliver_fn(int schedule, bool bf16) {
    if (schedule == 1) return bf16 ? (const void*)k_deliver_thread<true> : (const void*)k_deliver_thread<false>;
    return bf16 ? (const void*)k_deliver_warp<true> : (const void*)k_deliver_warp<false>;
}

// Persistent grid: as many blocks as fit on all SMs at once.
int deliver_default_grid(int schedule, int block, uint32_t nb, bool bf16) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = deliver_smem(nb, block);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, deliver_fn(schedule, bf16), block, smem);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

cudaError_t prepare_deliver(uint32_t nb) {
    const size_t smem = deliver_smem(nb, 1024);
    if (smem <= 48 * 1024) return cudaSuccess;
    for (int sch = 0; sch < 2; ++sch)
        for (int b = 0; b < 2; ++b) {
            cudaError_t e = cudaFuncSetAttribute(deliver_fn(sch, b != 0),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t launch_deliver(const NetView& v, int schedule, int block, int grid, cudaStream_t s) {
    const size_t smem = deliver_smem(v.nb, block);
    const bool bf16 = v.w_bf16 != 0;
    if (schedule == 1) {
        if (bf16)
            k_deliver_thread<true><<<grid, block, smem, s>>>(v);
        else
            k_deliver_thread<false><<<grid, block, smem, s>>>(v);
    } else {
        if (bf16)
            k_deliver_warp<true><<<grid, block, smem, s>>>(v);
        else
            k_deliver_warp<false><<<grid, block, smem, s>>>(v);
    }
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace snn
