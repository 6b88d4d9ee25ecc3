// shard_kernels.cu -- one time step of a shard of a spatially decomposed network.
//
// The paper distributes a network over processes that each own a tile of
// cortical modules (Sec. II-D): every process integrates its own neurons,
// tells the processes whose tiles its spikes can reach how many spikes it
// has and then which (the two-step exchange, Sec. II-E), and each process
// expands the spikes it receives into synaptic events with its own copy of
// the synapses that target it (deferred arborization, Sec. II-C).  Here a
// shard owns a stripe of module rows:
//   k_shard_neurons  the stripe's neurons (the update of every other
//                    schedule: ring slot, Poisson drive, Eq. 1-2, threshold,
//                    reset, refractory, adaptation), one spike bit each;
//   k_shard_compact  the spike bits into the outbox (global ids, increasing)
//                    and the shard's raster, one CTA;
//   k_shard_deliver  the inbound spike lists (the shard's own outbox and its
//                    peers') through the target-side table into the shard's
//                    delay ring, one warp per spike.
// The same integer sums as the single-network kernels: results are identical.
#include "device_common.cuh"

namespace snn {

constexpr int SHARD_THREADS = 256;
constexpr int SHARD_COMPACT_THREADS = 1024;

__global__ void __launch_bounds__(SHARD_THREADS) k_shard_neurons(NetView v, ShardView sv, uint32_t t) {
    __shared__ uint32_t s_pois[MAX_POIS];
    load_poisson_table(v, s_pois);
    __syncthreads();
    const uint32_t li = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    bool spike = false;
    uint32_t n_ext = 0;
    if (li < sv.Nl) {
        const uint32_t i = sv.n0 + li;
        int32_t* slot = sv.ring + (size_t)(t % v.D) * sv.Nlpad + li;
        const int32_t Ir = *slot;
        *slot = 0;
        const U4 u = philox4x32_10(i, t, TAG_DRIVE, 0u, v.key0, v.key1);
        n_ext = poisson_count(s_pois, v.pois_pad, u.x);
        const bool forced = (uint64_t)u.y < v.imposed_thresh;
        const int32_t I = (int32_t)((uint32_t)Ir + n_ext * (uint32_t)v.J_ext_fx);
        float V = sv.V[li], c = sv.c[li];
        uint32_t r = sv.ref[li];
        spike = lif_update(v, V, c, r, (i % v.M) < v.n_exc, I, forced);
        sv.V[li] = V;
        sv.c[li] = c;
        sv.ref[li] = (uint8_t)r;
    }
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, spike);
    if (lane == 0 && li < sv.Nl) sv.spk_bits[li >> 5] = bits;
    unsigned long long e = n_ext;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    if (lane == 0 && e) atomicAdd(reinterpret_cast<unsigned long long*>(&sv.cnt->ext_events), e);
}

__global__ void __launch_bounds__(SHARD_COMPACT_THREADS) k_shard_compact(ShardView sv, uint32_t t, uint32_t K) {
    __shared__ uint32_t s_w[SHARD_COMPACT_THREADS / 32];
    __shared__ unsigned long long s_rc;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_rc = sv.cnt->raster_count;
    __syncthreads();
    const uint64_t rc = s_rc;
    const uint32_t words = (sv.Nl + 31) >> 5;
    uint32_t run = 0;
    for (uint32_t base = 0; base < words; base += SHARD_COMPACT_THREADS) {
        const uint32_t w = base + threadIdx.x;
        uint32_t bits = w < words ? sv.spk_bits[w] : 0u;
        const uint32_t cnt = __popc(bits);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (uint32_t k = 0; k < SHARD_COMPACT_THREADS / 32; ++k) {
            before += k < warp ? s_w[k] : 0u;
            total += s_w[k];
        }
        uint32_t pos = run + before + incl - cnt;
        while (bits) {
            const uint32_t b = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint32_t id = sv.n0 + (w << 5) + b;
            sv.out_ids[pos] = id;
            const uint64_t r = rc + pos;
            if (r < sv.raster_cap) {
                sv.raster_t[r] = t;
                sv.raster_id[r] = id;
            }
            ++pos;
        }
        run += total;
        __syncthreads();  // s_w is rewritten by the next tile
    }
    if (threadIdx.x == 0) {
        *sv.out_cnt = run;
        sv.cnt->raster_count = rc + run;
        sv.cnt->n_spikes += run;
        sv.cnt->rec_events += (unsigned long long)run * K;
    }
}

template <bool BF16>
__global__ void __launch_bounds__(SHARD_THREADS) k_shard_deliver(NetView v, ShardView sv, ShardInbound in, uint32_t t) {
    __shared__ uint32_t s_pre[SHARD_MAX_LISTS + 1];
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (uint32_t l = 0; l < in.n; ++l) {
            s_pre[l] = acc;
            acc += *in.cnt[l];
        }
        s_pre[in.n] = acc;
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t total = s_pre[in.n];
    for (uint32_t j = gw; j < total; j += nw) {  // warp-uniform
        uint32_t l = 0;
        while (l + 1 < in.n && s_pre[l + 1] <= j) ++l;
        const uint32_t id = __ldcg(in.ids[l] + (j - s_pre[l]));
        const uint32_t r = id - sv.h0;
        if (r >= sv.rows) continue;  // a source outside the halo reaches nothing here
        const uint64_t a = __ldg(sv.row_ptr + r), e = __ldg(sv.row_ptr + r + 1);
        for (uint64_t k = a + lane; k < e; k += 32) {
            const uint32_t x = __ldg(sv.td + k);
            const float w = BF16 ? __uint_as_float((uint32_t)__ldg(reinterpret_cast<const uint16_t*>(sv.w) + k) << 16)
                                 : __ldg(reinterpret_cast<const float*>(sv.w) + k);
            uint32_t s = t % v.D + (x >> 24);
            if (s >= v.D) s -= v.D;
            red_add(sv.ring + (size_t)s * sv.Nlpad + (x & 0xFFFFFFu), fx_weight(v, w));
        }
    }
}

cudaError_t launch_shard_step(const NetView& v, const ShardView& sv, uint32_t t, cudaStream_t s) {
    if (sv.Nl > 0) {
        k_shard_neurons<<<(sv.Nl + SHARD_THREADS - 1) / SHARD_THREADS, SHARD_THREADS, 0, s>>>(v, sv, t);
        count_launch(1);
    }
    k_shard_compact<<<1, SHARD_COMPACT_THREADS, 0, s>>>(sv, t, v.K);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_shard_deliver(const NetView& v, const ShardView& sv, const ShardInbound& in, uint32_t t,
                                 cudaStream_t s) {
    if (in.n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = 4 * (sms > 0 ? sms : 1);
    if (v.w_bf16)
        k_shard_deliver<true><<<grid, SHARD_THREADS, 0, s>>>(v, sv, in, t);
    else
        k_shard_deliver<false><<<grid, SHARD_THREADS, 0, s>>>(v, sv, in, t);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace snn
