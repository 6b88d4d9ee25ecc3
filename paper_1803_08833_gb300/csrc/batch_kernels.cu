// batch_kernels.cu -- many independent networks advanced in one cooperative launch.
//
// All networks share one global index space of neuron quads and, every step,
// one global space of delivery tasks; both are split evenly over all warps
// of the grid, so small and large networks, sparse and busy ones, are
// balanced together behind one pair of grid barriers per step.  Network k
// owns quads [qoff[k], qoff[k+1]); warp wg owns global quads
// [Qtot wg / TW, Qtot (wg+1) / TW), which may cover parts of several
// networks.  For every (network, warp) segment the warp compacts that
// network's spikes in id order into the network's staging array and records
// their count, so each network keeps its (step, id) spike order and its
// results are bit-identical to running it alone.
#include "grid_common.cuh"

namespace snn {

// Launch shapes of the global layout (snn_batch_set_shape): shape 0 runs two
// CTAs per SM with four delivery tasks in flight per warp (many small
// networks need more warps than deep unrolling), shape 1 one CTA per SM with
// six (the single-network persistent kernel's shape).
template <int SHAPE>
struct BatchShape;
template <>
struct BatchShape<0> {
    static constexpr int MIN_BLOCKS = 2, UNROLL = 4;
};
template <>
struct BatchShape<1> {
    static constexpr int MIN_BLOCKS = 1, UNROLL = 6;
};

// Neuron id of spike jl of network k: the (network, warp) segment by binary
// search over the network's part of the segment prefix, then the warp's
// staging area.
__device__ __forceinline__ uint32_t batch_spike_id(const BatchMeta& bm, const uint32_t* s_wpre, const uint32_t* s_cbase,
                                                   const uint32_t* s_qoff, uint32_t k, uint32_t jl, uint32_t TW) {
    const uint32_t base = s_cbase[k], cnt = s_cbase[k + 1] - base, pre0 = s_wpre[base];
    uint32_t lo = 0, hi = cnt;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_wpre[base + mid] - pre0 <= jl)
            lo = mid;
        else
            hi = mid;
    }
    const uint32_t wg = bm.wlo[k] + lo;
    const uint32_t A = (uint32_t)((uint64_t)bm.Qtot * wg / TW);
    const uint32_t qa = max(A, s_qoff[k]) - s_qoff[k];
    return __ldcg(bm.views[k].seg + ((size_t)qa << 2) + (jl - (s_wpre[base + lo] - pre0)));
}

// Largest k with pre[k] <= x (pre nondecreasing, pre[0] <= x).
__device__ __forceinline__ uint32_t upper_slot(const uint32_t* pre, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <int SHAPE>
__global__ void __launch_bounds__(PERSIST_THREADS, BatchShape<SHAPE>::MIN_BLOCKS)
    k_run_batch(BatchMeta bm, uint32_t n_steps) {
    constexpr int BATCH_UNROLL = BatchShape<SHAPE>::UNROLL;  // delivery tasks in flight per warp
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t n = bm.n, NW = bm.n_seg;
    const uint32_t G = gridDim.x, TW = G * PERSIST_WARPS;
    unsigned long long* s_rc = reinterpret_cast<unsigned long long*>(smem);  // n raster counters
    unsigned long long* s_spk = s_rc + n;                                     // n spike totals (this launch)
    uint32_t* s_qoff = reinterpret_cast<uint32_t*>(s_spk + n);               // n + 1
    uint32_t* s_cbase = s_qoff + n + 1;                                        // n + 1
    uint32_t* s_spre = s_cbase + n + 1;                                        // n + 1 spike prefix
    uint32_t* s_tpre = s_spre + n + 1;                                         // n + 1 task prefix
    uint32_t* s_t0 = s_tpre + n + 1;                                           // n
    uint32_t* s_steps = s_t0 + n;                                              // n
    uint32_t* s_wpre = s_steps + n;                                            // NW + 1
    uint32_t* s_id = s_wpre + NW + 1;                                          // PERSIST_THREADS
    for (uint32_t k = threadIdx.x; k <= n; k += blockDim.x) {
        s_qoff[k] = bm.qoff[k];
        s_cbase[k] = bm.cbase[k];
        if (k < n) {
            s_t0[k] = bm.views[k].st->t;
            s_rc[k] = bm.views[k].st->raster_count;
            s_spk[k] = 0;
            s_steps[k] = bm.steps[k];
        }
    }
    uint32_t gen = 0;  // barriers passed in this launch
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wg = blockIdx.x * PERSIST_WARPS + warp;
    const uint32_t A = (uint32_t)((uint64_t)bm.Qtot * wg / TW);
    const uint32_t B = (uint32_t)((uint64_t)bm.Qtot * (wg + 1) / TW);
    const uint64_t pol = evict_first_policy();
    uint32_t done = 0;
    bool ok = true;

    for (uint32_t step = 0; step < n_steps; ++step) {
        // ---- phase N: every (network, warp) segment of this warp
        if (A < B) {
            uint32_t k = upper_slot(s_qoff, n, A);
            for (uint32_t q0 = A; q0 < B; ++k) {
                while (s_qoff[k + 1] <= q0) ++k;  // skip networks without quads
                const uint32_t qe = min(B, s_qoff[k + 1]);
                const NetView& v = bm.views[k];
                uint32_t run = 0;
                if (step < s_steps[k]) {
                    const uint32_t t = s_t0[k] + step;
                    const uint32_t slot = t % v.D;
                    const uint32_t qa = q0 - s_qoff[k], qb = qe - s_qoff[k];
                    uint32_t ext = 0;
                    uint64_t rec = 0;
                    for (uint32_t qc = qa; qc < qb; qc += 32) {
                        const uint32_t q = qc + lane;
                        uint32_t spk = 0;
                        if (q < qb) spk = update_quad(v, v.pois32, q << 2, t, slot, ext, rec);
                        const uint32_t cnt = __popc(spk);
                        uint32_t incl = cnt;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                            if (lane >= (uint32_t)o) incl += y;
                        }
                        uint32_t pos = (qa << 2) + run + incl - cnt;
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if (spk & (1u << b)) v.seg[pos++] = (q << 2) + b;
                        run += __shfl_sync(0xFFFFFFFFu, incl, 31);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) ext += __shfl_xor_sync(0xFFFFFFFFu, ext, o);
                    if (lane == 0 && ext) atomicAdd(reinterpret_cast<unsigned long long*>(&v.st->ext_events),
                                                    (unsigned long long)ext);
                    if (v.row_len) {  // pairwise rule: recurrent events are the spiking rows' lengths
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) rec += __shfl_xor_sync(0xFFFFFFFFu, rec, o);
                        if (lane == 0 && rec) atomicAdd(reinterpret_cast<unsigned long long*>(&v.st->rec_events),
                                                        (unsigned long long)rec);
                    }
                }
                if (lane == 0) bm.wcnt[s_cbase[k] + (wg - bm.wlo[k])] = run;
                q0 = qe;
            }
        }
        if (!grid_barrier_on(bm.bst, G + bm.barrier_extra, bm.wait_limit_ns, gen)) {
            ok = false;
            break;
        }

        // ---- phase D: per-network spike and task offsets
        block_exclusive_scan(bm.wcnt, NW, s_wpre);
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
            const uint32_t S = step < s_steps[k] ? s_wpre[s_cbase[k + 1]] - s_wpre[s_cbase[k]] : 0u;
            s_spre[k] = S;
            s_tpre[k] = S * ((bm.views[k].K + 127) >> 7);
        }
        __syncthreads();
        block_scan_inplace(s_spre, n);
        block_scan_inplace(s_tpre, n);
        // raster entries of every network
        const uint32_t total = s_spre[n];
        for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += G * blockDim.x) {
            const uint32_t k = upper_slot(s_spre, n, j);
            const uint32_t jl = j - s_spre[k];
            const NetView& v = bm.views[k];
            const uint64_t r = s_rc[k] + jl;
            if (r < v.raster_cap) {
                v.raster_t[r] = s_t0[k] + step;
                v.raster_id[r] = batch_spike_id(bm, s_wpre, s_cbase, s_qoff, k, jl, TW);
            }
        }
        // this CTA's share of the global task space
        const uint64_t T = s_tpre[n];
        uint64_t ta = T * blockIdx.x / G;
        const uint64_t tb = T * (blockIdx.x + 1) / G;
        if (ta < tb) {
            for (uint32_t k = upper_slot(s_tpre, n, (uint32_t)ta); ta < tb; ++k) {
                if (s_tpre[k + 1] <= ta) continue;
                const NetView& v = bm.views[k];
                const uint32_t chunks = (v.K + 127) >> 7;
                const uint64_t la = ta - s_tpre[k];
                const uint64_t lb = min(tb, (uint64_t)s_tpre[k + 1]) - s_tpre[k];
                const uint32_t slot0 = (s_t0[k] + step) % v.D;
                const uint32_t j_last = (uint32_t)((lb - 1) / chunks);
                const bool bf16 = v.w_bf16 != 0;
                for (uint32_t jb = (uint32_t)(la / chunks); jb <= j_last; jb += blockDim.x) {
                    const uint32_t j = jb + threadIdx.x;
                    if (j <= j_last) s_id[threadIdx.x] = batch_spike_id(bm, s_wpre, s_cbase, s_qoff, k, j, TW);
                    __syncthreads();
                    const uint64_t lo = max(la, (uint64_t)jb * chunks);
                    const uint64_t hi = min(lb, (uint64_t)(jb + blockDim.x) * chunks);
                    for (uint64_t tk = lo + warp; tk < hi; tk += (uint64_t)PERSIST_WARPS * BATCH_UNROLL) {
                        if (bf16)
                            deliver_tasks<true, BATCH_UNROLL>(v, tk, PERSIST_WARPS, hi, chunks, s_id, jb, slot0, lane,
                                                              pol);
                        else
                            deliver_tasks<false, BATCH_UNROLL>(v, tk, PERSIST_WARPS, hi, chunks, s_id, jb, slot0, lane,
                                                               pol);
                    }
                    __syncthreads();
                }
                ta = s_tpre[k + 1];
            }
        }
        // every thread of the CTA is past its raster writes (which read s_rc) before
        // the counters move on; a CTA without delivery tasks has no barrier in between
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
            const uint32_t S = s_spre[k + 1] - s_spre[k];
            s_rc[k] += S;
            s_spk[k] += S;
        }
        if (!grid_barrier_on(bm.bst, G + bm.barrier_extra, bm.wait_limit_ns, gen)) {
            ok = false;
            break;
        }
        done = step + 1;
    }

    if (blockIdx.x == 0) {
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
            DevState* st = bm.views[k].st;
            if (!ok) {
                atomicOr(&st->err, ERR_BARRIER_TIMEOUT);
                continue;
            }
            st->t = s_t0[k] + min(s_steps[k], done);
            st->raster_count = s_rc[k];
            st->n_spikes += s_spk[k];
            if (!bm.views[k].row_len) st->rec_events += s_spk[k] * bm.views[k].K;
            st->n_spk = 0;
        }
    }
}

static size_t batch_smem(uint32_t n, uint32_t n_seg) {
    return (size_t)n * 16 + (size_t)(4 * (n + 1) + 2 * n + n_seg + 1 + PERSIST_THREADS) * sizeof(uint32_t);
}

static const void* batch_fn(int shape) {
    return shape == 1 ? (const void*)k_run_batch<1> : (const void*)k_run_batch<0>;
}

int batch_grid(uint32_t n, uint32_t n_seg_bound, int shape) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = batch_smem(n, n_seg_bound);
    const void* fn = batch_fn(shape);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, PERSIST_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return fit * sms;
}

cudaError_t launch_batch(const BatchMeta& bm, uint32_t n_steps, int grid, int shape, cudaStream_t s) {
    const size_t smem = batch_smem(bm.n, bm.n_seg);
    const void* fn = batch_fn(shape);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    BatchMeta m = bm;
    uint32_t ns = n_steps;
    void* args[] = {&m, &ns};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(PERSIST_THREADS), args, smem, s);
    count_launch(1);
    return e;
}

}  // namespace snn
