// stdp_kernels.cu -- spike-timing dependent plasticity (Sec. II-A).
//
// The paper computes STDP contributions when a neuron spikes (flow step 1)
// and when a spike arrives at a synapse (flow step 4), and every second
// integrates them into a long-term change applied to each synapse.  This
// build's rule (the paper gives none): pair-based with exponential traces,
// excitatory synapses only.  Per step t, after the neuron kernel and before
// the delivery of the step's spikes:
//   k_stdp_decay  x(t-1) into the history, then y *= a_minus, x *= a_plus
//                 for every neuron (x: pre-synaptic trace, y: post-synaptic);
//   k_stdp_post   y += 1, x += 1 for the step's spikes; the step's spike list
//                 into the history ring (slot t mod D);
//   k_stdp_ltd    every arrival of step t -- synapse k of a spike of step
//                 t - d with delay d, found by walking the rows of the last
//                 D - 1 steps' spikes -- loses A_minus y_target(t);
//   k_stdp_ltp    every synapse into a neuron that spiked at t (a
//                 target-major index) gains A_plus x_source(t - d - 1) a_plus,
//                 the trace of its arrivals strictly before t;
// and after the delivery, k_stdp_apply adds the accumulated change to the
// excitatory weights (clipped to [0, w_max]) at the end of every period.
// Contributions are rounded once to the 2^-16 mV grid and summed in int32:
// the order of the sums never matters.
#include "device_common.cuh"

#include <algorithm>

namespace snn {

constexpr int STDP_THREADS = 256;

__device__ __forceinline__ int32_t stdp_fx(float c) { return __float2int_rn(__fmul_rn(c, 65536.0f)); }

__global__ void k_stdp_decay(NetView v, StdpView p) {
    const uint32_t t = v.st->t_deliver;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    const float x = p.x[i];
    if (t >= 1) p.xh[(size_t)((t - 1) % (v.D + 1)) * v.Npad + i] = x;
    p.y[i] = __fmul_rn(p.y[i], p.a_minus);
    p.x[i] = __fmul_rn(x, p.a_plus);
}

// Id of staged spike j of the step (the per-block staging of k_neuron_step).
__device__ __forceinline__ uint32_t staged_spike(const NetView& v, uint32_t j) {
    uint32_t lo = 0, hi = v.nb;  // largest block b with blk_off[b] <= j
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldcg(v.blk_off + mid) <= j)
            lo = mid;
        else
            hi = mid;
    }
    return __ldcg(v.seg + (size_t)lo * NEURONS_PER_BLOCK + (j - __ldcg(v.blk_off + lo)));
}

__global__ void k_stdp_post(NetView v, StdpView p) {
    const uint32_t t = v.st->t_deliver, n_spk = v.st->n_spk;
    const uint32_t slot = t % v.D;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_spk; j += stride) {
        const uint32_t id = staged_spike(v, j);
        p.y[id] = __fadd_rn(p.y[id], 1.0f);
        p.x[id] = __fadd_rn(p.x[id], 1.0f);
        p.hist[(size_t)slot * v.Npad + j] = id;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) p.hist_cnt[slot] = n_spk;
}

// One warp per (delay d, spike of step t - d); its row's synapses with delay d
// arrive now.
__global__ void k_stdp_ltd(NetView v, StdpView p) {
    const uint32_t t = v.st->t_deliver;
    __shared__ uint32_t s_pre[256 + 1];  // spikes of steps t - 1 .. t - (D - 1), prefix
    const uint32_t dmax = min(v.D - 1, t);
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (uint32_t d = 1; d <= dmax; ++d) {
            s_pre[d - 1] = acc;
            acc += __ldcg(p.hist_cnt + (t - d) % v.D);
        }
        s_pre[dmax] = acc;
    }
    __syncthreads();
    const uint32_t total = s_pre[dmax];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = gw; q < total; q += nw) {  // warp-uniform
        uint32_t d = 1;
        while (d < dmax && s_pre[d] <= q) ++d;
        const uint32_t src = __ldcg(p.hist + (size_t)((t - d) % v.D) * v.Npad + (q - s_pre[d - 1]));
        if (src % v.M >= v.n_exc) continue;  // inhibitory synapses are not plastic
        const uint32_t L = v.row_len ? __ldg(v.row_len + src) : v.K;
        const size_t row = (size_t)src * v.Kpad;
        for (uint32_t k = lane; k < L; k += 32) {
            const uint32_t x = __ldg(v.td + row + k);
            if ((x >> 24) != d) continue;
            const float c = __fmul_rn(p.A_minus, __ldcg(p.y + (x & 0xFFFFFFu)));
            p.delta[row + k] -= stdp_fx(c);
        }
    }
}

// One warp per spike of step t; its incoming synapses gain.
__global__ void k_stdp_ltp(NetView v, StdpView p) {
    const uint32_t t = v.st->t_deliver;
    const uint32_t slot = t % v.D;
    const uint32_t n_spk = __ldcg(p.hist_cnt + slot);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t j = gw; j < n_spk; j += nw) {  // warp-uniform
        const uint32_t post = __ldcg(p.hist + (size_t)slot * v.Npad + j);
        const uint64_t a = __ldg(p.in_ptr + post), b = __ldg(p.in_ptr + post + 1);
        for (uint64_t q = a + lane; q < b; q += 32) {
            const uint64_t e = __ldg(p.in_syn + q);
            const uint32_t src = (uint32_t)(e / v.Kpad);
            if (src % v.M >= v.n_exc) continue;
            const uint32_t d = __ldg(v.td + e) >> 24;
            if (t < d + 1) continue;  // no arrival can precede the start
            const float xa = __fmul_rn(__ldcg(p.xh + (size_t)((t - d - 1) % (v.D + 1)) * v.Npad + src), p.a_plus);
            p.delta[e] += stdp_fx(__fmul_rn(p.A_plus, xa));
        }
    }
}

// At the end of every period: w <- clip(w + delta 2^-16, 0, w_max), delta <- 0.
__global__ void k_stdp_apply(NetView v, StdpView p) {
    const uint32_t t = v.st->t_deliver;
    if ((t + 1) % p.period != 0) return;
    const uint64_t n = (uint64_t)v.N * v.Kpad;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    float* w = reinterpret_cast<float*>(v.w);
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const uint32_t src = (uint32_t)(e / v.Kpad);
        if (src % v.M >= v.n_exc) continue;
        const uint32_t k = (uint32_t)(e - (uint64_t)src * v.Kpad);
        const uint32_t L = v.row_len ? __ldg(v.row_len + src) : v.K;
        if (k >= L) continue;
        float nw = __fadd_rn(w[e], __fmul_rn(__int2float_rn(p.delta[e]), 1.0f / 65536.0f));
        nw = nw < 0.0f ? 0.0f : nw;
        nw = nw > p.w_max ? p.w_max : nw;
        w[e] = nw;
        p.delta[e] = 0;
    }
}

// Incoming index: counts per target, then (after a host scan) the synapse
// indices e = source * Kpad + k of every target's incoming synapses.
__global__ void k_stdp_in_count(NetView v, uint64_t* cnt) {
    const uint64_t n = (uint64_t)v.N * v.Kpad;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const uint32_t src = (uint32_t)(e / v.Kpad), k = (uint32_t)(e - (uint64_t)src * v.Kpad);
        const uint32_t L = v.row_len ? __ldg(v.row_len + src) : v.K;
        if (k < L) atomicAdd(reinterpret_cast<unsigned long long*>(cnt + (__ldg(v.td + e) & 0xFFFFFFu)), 1ull);
    }
}

__global__ void k_stdp_in_fill(NetView v, uint64_t* cursor, uint64_t* in_syn) {
    const uint64_t n = (uint64_t)v.N * v.Kpad;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const uint32_t src = (uint32_t)(e / v.Kpad), k = (uint32_t)(e - (uint64_t)src * v.Kpad);
        const uint32_t L = v.row_len ? __ldg(v.row_len + src) : v.K;
        if (k < L) {
            const uint64_t pos = atomicAdd(reinterpret_cast<unsigned long long*>(cursor + (__ldg(v.td + e) & 0xFFFFFFu)), 1ull);
            in_syn[pos] = e;
        }
    }
}

static int stdp_grid(uint64_t work) {
    const uint64_t b = (work + STDP_THREADS - 1) / STDP_THREADS;
    return (int)std::min<uint64_t>(std::max<uint64_t>(b, 1), 4096);
}

cudaError_t launch_stdp_index(const NetView& v, uint64_t* cnt_or_cursor, uint64_t* in_syn, cudaStream_t s) {
    const int g = stdp_grid((uint64_t)v.N * v.Kpad);
    if (in_syn)
        k_stdp_in_fill<<<g, STDP_THREADS, 0, s>>>(v, cnt_or_cursor, in_syn);
    else
        k_stdp_in_count<<<g, STDP_THREADS, 0, s>>>(v, cnt_or_cursor);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_stdp_pre_delivery(const NetView& v, const StdpView& p, cudaStream_t s) {
    k_stdp_decay<<<(v.N + STDP_THREADS - 1) / STDP_THREADS, STDP_THREADS, 0, s>>>(v, p);
    k_stdp_post<<<stdp_grid(v.N), STDP_THREADS, 0, s>>>(v, p);
    k_stdp_ltd<<<stdp_grid((uint64_t)v.N * 32), STDP_THREADS, 0, s>>>(v, p);
    k_stdp_ltp<<<stdp_grid((uint64_t)v.N * 32), STDP_THREADS, 0, s>>>(v, p);
    count_launch(4);
    return cudaGetLastError();
}

cudaError_t launch_stdp_apply(const NetView& v, const StdpView& p, cudaStream_t s) {
    k_stdp_apply<<<stdp_grid((uint64_t)v.N * v.Kpad), STDP_THREADS, 0, s>>>(v, p);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace snn
