// build_kernels.cu -- construction phase (Sec. II-A phase 1, Sec. II-B, Sec. III-B).
//
//   k_build_cdf    per source module: FP64 lateral-kernel values over the in-grid
//                  modules of the cut-off disc, their normalisation (the A / B
//                  constants of Sec. I and Sec. III-B) and cumulative distribution,
//                  converted to uint32 thresholds.
//   k_gen_synapses per (neuron, 4 synapses): Philox draws -> target module by
//                  inverse CDF, target neuron, weight, delay; 16 B vector stores
//                  of target | delay << 24 and of the weights.
//   k_pair_count / k_pair_rows / k_pair_fill / k_pair_attr
//                  the pairwise law of Sec. III-B: per (neuron, stencil entry)
//                  the connection draws of every candidate target, counted,
//                  turned into row offsets, then written.
//   k_init_state   V = V_th * U[0,1), c = 0, ref = 0.
//
// Floating point is written with explicit round-to-nearest intrinsics, so no
// multiply-add is ever contracted: the tables and weights are reproducible
// bit for bit by any IEEE implementation of the same expressions.
#include "philox.cuh"
#include "snn_internal.h"

#include <cuda_bf16.h>

namespace snn {

// Kernel value of one grid offset with squared grid distance d2.
__device__ __forceinline__ double lateral_kernel(const BuildView& b, uint32_t d2) {
    const double dd = (double)d2;
    if (b.kernel == 0) {
        // Gaussian B exp(-r^2 / 2 sigma^2), r^2 = d2 * spacing^2
        const double num = __dmul_rn(__dmul_rn(dd, b.spacing), b.spacing);
        const double den = __dmul_rn(__dmul_rn(2.0, b.sigma), b.sigma);
        return exp(-__ddiv_rn(num, den));
    }
    // exponential A exp(-r / lambda), r = spacing * sqrt(d2)
    const double r = __dmul_rn(b.spacing, __dsqrt_rn(dd));
    return exp(-__ddiv_rn(r, b.lambda));
}

// One block per source module.  Threads evaluate the kernel of every offset
// in parallel; one thread then accumulates the in-grid values in the fixed
// (dy, dx) order (a sequential FP64 sum, so the rounding is reproducible);
// finally threads convert cdf = prefix / total to thresholds floor(cdf 2^32).
__global__ void __launch_bounds__(256) k_build_cdf(BuildView b) {
    const uint32_t m = blockIdx.x;
    const int sx = (int)(m % b.grid_w), sy = (int)(m / b.grid_w);
    double* f = b.scratch + (size_t)m * b.max_off;
    for (uint32_t j = threadIdx.x; j < b.max_off; j += blockDim.x) {
        const int dx = b.offsets[2 * j], dy = b.offsets[2 * j + 1];
        const int tx = sx + dx, ty = sy + dy;
        const bool in = tx >= 0 && ty >= 0 && tx < (int)b.grid_w && ty < (int)b.grid_h;
        f[j] = in ? lateral_kernel(b, (uint32_t)(dx * dx + dy * dy)) : -1.0;
    }
    __syncthreads();
    __shared__ uint32_t s_n;
    __shared__ double s_total;
    if (threadIdx.x == 0) {
        uint32_t n = 0;
        double P = 0.0;
        uint32_t* tm = b.cdf_mod + (size_t)m * b.max_off;
        for (uint32_t j = 0; j < b.max_off; ++j) {
            const double v = f[j];
            if (v < 0.0) continue;
            P = __dadd_rn(P, v);
            f[n] = P;  // n <= j: compacting in place never overwrites an unread value
            const int dx = b.offsets[2 * j], dy = b.offsets[2 * j + 1];
            tm[n] = (uint32_t)(sy + dy) * b.grid_w + (uint32_t)(sx + dx);
            ++n;
        }
        s_n = n;
        s_total = P;
        b.cdf_n[m] = n;
    }
    __syncthreads();
    const uint32_t n = s_n;
    const double S = s_total;
    uint32_t* T = b.cdf_T + (size_t)m * b.max_off;
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
        uint32_t th = 0xFFFFFFFFu;
        if (j + 1 < n) {
            const double x = floor(__dmul_rn(__ddiv_rn(f[j], S), 4294967296.0));
            th = x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
        }
        T[j] = th;
    }
}

// Number of thresholds <= u among the first n - 1 entries: the index of the
// first entry with u < T (inverse-CDF sampling of the target module).
__device__ __forceinline__ uint32_t upper_index(const uint32_t* __restrict__ T, uint32_t n, uint32_t u) {
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(T + mid) <= u)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Efficacy and delay of a synapse from words u2 and u3 of its Philox block
// (Sec. II-B): uniform or Gaussian-quantile efficacy, uniform or truncated
// exponential delay; inhibitory delays are constant.
__device__ __forceinline__ void syn_attr(const BuildView& b, bool exc, uint32_t u2, uint32_t u3, float& w, uint32_t& d) {
    if (exc) {
        w = b.weight_dist ? __ldg(b.wtab + (u2 >> 20)) : __fadd_rn(b.w_lo, __fmul_rn(b.w_span, unit24(u2)));
        if (b.delay_dist) {
            uint32_t k = 0;
            for (uint32_t j = 0; j < b.n_dthr; ++j) k += __ldg(b.dthr + j) <= (uint64_t)u3 ? 1u : 0u;
            d = b.d_lo + k;
        } else {
            d = b.d_lo + __umulhi(u3, b.d_span);
        }
    } else {
        w = b.weight_dist ? __ldg(b.wtab + WTAB + (u2 >> 20)) : b.w_inh;
        d = b.d_inh;
    }
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_gen_synapses(BuildView b, uint32_t* __restrict__ td,
                                                      void* __restrict__ wout) {
    const uint32_t groups = b.Kpad >> 2;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)b.N * groups) return;
    const uint32_t i = (uint32_t)(gid / groups);
    const uint32_t k0 = (uint32_t)(gid - (uint64_t)i * groups) << 2;
    const uint32_t s = i / b.M;
    const bool exc = (i - s * b.M) < b.n_exc;
    const uint32_t* T = b.cdf_T + (size_t)s * b.max_off;
    const uint32_t* TM = b.cdf_mod + (size_t)s * b.max_off;
    const uint32_t n = __ldg(b.cdf_n + s);
    uint32_t tg[4];
    float w[4];
    uint32_t d[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t k = k0 + q;
        tg[q] = 0;
        w[q] = 0.0f;
        d[q] = 0;
        if (k < b.K) {
            const U4 u = philox4x32_10(i, k, TAG_GEN, 0u, b.key0, b.key1);
            const uint32_t j = upper_index(T, n, u.x);
            tg[q] = __ldg(TM + j) * b.M + __umulhi(u.y, b.M);
            syn_attr(b, exc, u.z, u.w, w[q], d[q]);
        }
    }
    const size_t e = (size_t)i * b.Kpad + k0;
    *reinterpret_cast<uint4*>(td + e) =
        make_uint4(tg[0] | (d[0] << 24), tg[1] | (d[1] << 24), tg[2] | (d[2] << 24), tg[3] | (d[3] << 24));
    if (BF16) {
        __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(wout) + e;
        __nv_bfloat162 a = __halves2bfloat162(__float2bfloat16_rn(w[0]), __float2bfloat16_rn(w[1]));
        __nv_bfloat162 c = __halves2bfloat162(__float2bfloat16_rn(w[2]), __float2bfloat16_rn(w[3]));
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&a);
        pk.y = *reinterpret_cast<uint32_t*>(&c);
        *reinterpret_cast<uint2*>(wb) = pk;
    } else {
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(wout) + e) = make_float4(w[0], w[1], w[2], w[3]);
    }
}

// Synapse (i, k): target, weight, delay and stencil index j of its target module.
struct Draw {
    uint32_t tgt, j, d;
    float w;
};

__device__ __forceinline__ Draw draw_synapse(const BuildView& b, uint32_t i, uint32_t k, bool exc, const uint32_t* T,
                                             const uint32_t* TM, uint32_t n) {
    const U4 u = philox4x32_10(i, k, TAG_GEN, 0u, b.key0, b.key1);
    Draw r;
    r.j = upper_index(T, n, u.x);
    r.tgt = __ldg(TM + r.j) * b.M + __umulhi(u.y, b.M);
    syn_attr(b, exc, u.z, u.w, r.w, r.d);
    return r;
}

// Grouped layout: one warp per row.  Pass 1 counts the row's synapses per
// stencil entry j (shared-memory histogram) and writes the segment index
// (exclusive prefix; entry n_s = K).  Pass 2 redraws the synapses in k order,
// 32 at a time, and scatters each to cursor[j] + (its rank among the lanes of
// the same j), so every segment keeps the draw order: the row is the stable
// sort of the draw-order row by stencil index (= by target module).
template <bool BF16>
__global__ void __launch_bounds__(256) k_gen_grouped(BuildView b, uint32_t* __restrict__ td,
                                                     void* __restrict__ wout) {
    extern __shared__ uint32_t s_cur[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* cur = s_cur + warp * (b.max_off + 1);
    const uint32_t i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= b.N) return;  // warp-uniform
    const uint32_t s = i / b.M;
    const bool exc = (i - s * b.M) < b.n_exc;
    const uint32_t* T = b.cdf_T + (size_t)s * b.max_off;
    const uint32_t* TM = b.cdf_mod + (size_t)s * b.max_off;
    const uint32_t n = __ldg(b.cdf_n + s);
    for (uint32_t j = lane; j <= b.max_off; j += 32) cur[j] = 0;
    __syncwarp();
    for (uint32_t k = lane; k < b.K; k += 32) {
        const U4 u = philox4x32_10(i, k, TAG_GEN, 0u, b.key0, b.key1);
        atomicAdd(&cur[upper_index(T, n, u.x)], 1u);
    }
    __syncwarp();
    // exclusive prefix over the n bins, 32 at a time
    uint16_t* seg = b.segidx + (size_t)i * (b.max_off + 1);
    uint32_t run = 0;
    for (uint32_t j0 = 0; j0 < n; j0 += 32) {
        const uint32_t j = j0 + lane;
        const uint32_t x = j < n ? cur[j] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (j < n) {
            cur[j] = run + incl - x;
            seg[j] = (uint16_t)(run + incl - x);
        }
        run += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    for (uint32_t j = n + lane; j <= b.max_off; j += 32) seg[j] = (uint16_t)b.K;
    __syncwarp();
    const size_t row = (size_t)i * b.Kpad;
    for (uint32_t k0 = 0; k0 < b.K; k0 += 32) {
        const uint32_t k = k0 + lane;
        const bool active = k < b.K;
        Draw r{0u, 0xFFFFFFFFu, 0u, 0.0f};
        if (active) r = draw_synapse(b, i, k, exc, T, TM, n);
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, r.j);
        if (active) {
            const uint32_t pos = cur[r.j] + __popc(peers & ((1u << lane) - 1u));
            td[row + pos] = r.tgt | (r.d << 24);
            if (BF16)
                reinterpret_cast<__nv_bfloat16*>(wout)[row + pos] = __float2bfloat16_rn(r.w);
            else
                reinterpret_cast<float*>(wout)[row + pos] = r.w;
        }
        __syncwarp();
        if (active && lane == (uint32_t)(__ffs(peers) - 1)) cur[r.j] += __popc(peers);
        __syncwarp();
    }
    for (uint32_t k = b.K + lane; k < b.Kpad; k += 32) {  // padding entries
        td[row + k] = 0u;
        if (BF16)
            reinterpret_cast<__nv_bfloat16*>(wout)[row + k] = __float2bfloat16_rn(0.0f);
        else
            reinterpret_cast<float*>(wout)[row + k] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Pairwise law (Sec. III-B).  Stencil entry o of neuron i covers the target
// module at (sx + dx_o, sy + dy_o); candidate j of that module is connected
// when word j % 4 of Philox (i, o * ceil(M/4) + j / 4, CONN) is below the
// entry's threshold (never j = i: no autapse).  Inhibitory neurons keep only
// the local entry when inh_local_only is set.  The row lists the connections
// in (o, j) order; the k-th takes its efficacy and delay from Philox
// (i, k, GEN).

// Candidates of (i, o) that connect; with WRITE, writes their targets from
// row offset `start` on (k_pair_attr adds the delays and efficacies, one
// thread per synapse, so that no lane of the candidate loop waits on another
// lane's draws).  Returns the count.
template <bool WRITE>
__device__ __forceinline__ uint32_t pair_entry(const BuildView& b, uint32_t i, uint32_t o, uint32_t start,
                                               uint32_t* __restrict__ td) {
    const uint32_t s = i / b.M, a = i - s * b.M;
    const bool exc = a < b.n_exc;
    const int dx = __ldg(b.pair_dx + o), dy = __ldg(b.pair_dy + o);
    const bool local = dx == 0 && dy == 0;
    if (!exc && b.inh_local_only && !local) return 0;
    const int tx = (int)(s % b.grid_w) + dx, ty = (int)(s / b.grid_w) + dy;
    if (tx < 0 || ty < 0 || tx >= (int)b.grid_w || ty >= (int)b.grid_h) return 0;
    const uint32_t base = ((uint32_t)ty * b.grid_w + (uint32_t)tx) * b.M;
    const uint64_t thr = __ldg(b.pair_thr + o);
    const uint32_t c4 = (b.M + 3u) >> 2;
    uint32_t n = 0;
    for (uint32_t g = 0; g < c4; ++g) {
        const U4 u = philox4x32_10(i, o * c4 + g, TAG_CONN, 0u, b.key0, b.key1);
        const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t j = (g << 2) + q;
            if (j >= b.M || (local && j == a) || (uint64_t)uw[q] >= thr) continue;
            if (WRITE) td[(size_t)i * b.Kpad + start + n] = base + j;
            ++n;
        }
    }
    return n;
}

__global__ void __launch_bounds__(256) k_pair_count(BuildView b) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)b.N * b.pair_n) return;
    const uint32_t i = (uint32_t)(gid / b.pair_n), o = (uint32_t)(gid - (uint64_t)i * b.pair_n);
    const uint32_t n = pair_entry<false>(b, i, o, 0u, nullptr);
    b.pair_cnt[(size_t)i * (b.pair_n + 1) + o] = (uint16_t)min(n, 0xFFFFu);
}

// One warp per row: exclusive prefix of the entry counts (in place: the row
// offset of each entry; entry pair_n holds the row length, so the row is a
// segment index of stride pair_n + 1), the row length and the longest row.
__global__ void __launch_bounds__(256) k_pair_rows(BuildView b) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= b.N) return;  // warp-uniform
    uint16_t* c = b.pair_cnt + (size_t)i * (b.pair_n + 1);
    uint32_t run = 0;
    for (uint32_t o0 = 0; o0 < b.pair_n; o0 += 32) {
        const uint32_t o = o0 + lane;
        const uint32_t x = o < b.pair_n ? c[o] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, k);
            if (lane >= (uint32_t)k) incl += y;
        }
        if (o < b.pair_n) c[o] = (uint16_t)min(run + incl - x, 0xFFFFu);
        run += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) {
        b.row_len[i] = run;
        c[b.pair_n] = (uint16_t)min(run, 0xFFFFu);
        atomicMax(b.max_len, run);
    }
}

__global__ void __launch_bounds__(256) k_pair_fill(BuildView b, uint32_t* __restrict__ td) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)b.N * b.pair_n) return;
    const uint32_t i = (uint32_t)(gid / b.pair_n), o = (uint32_t)(gid - (uint64_t)i * b.pair_n);
    pair_entry<true>(b, i, o, b.pair_cnt[(size_t)i * (b.pair_n + 1) + o], td);
}

// Efficacy and delay of synapse k of row i from Philox (i, k, GEN), added to
// the target k_pair_fill wrote; four synapses per thread, rows of row_len[i].
template <bool BF16>
__global__ void __launch_bounds__(256) k_pair_attr(BuildView b, uint32_t* __restrict__ td, void* __restrict__ wout) {
    const uint32_t groups = b.Kpad >> 2;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (uint64_t)b.N * groups) return;
    const uint32_t i = (uint32_t)(gid / groups);
    const uint32_t k0 = (uint32_t)(gid - (uint64_t)i * groups) << 2;
    const uint32_t len = b.row_len[i];
    if (k0 >= len) return;
    const bool exc = (i % b.M) < b.n_exc;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t k = k0 + q;
        if (k < len) {
            const U4 u = philox4x32_10(i, k, TAG_GEN, 0u, b.key0, b.key1);
            float w;
            uint32_t d;
            syn_attr(b, exc, u.z, u.w, w, d);
            const size_t e = (size_t)i * b.Kpad + k;
            td[e] |= d << 24;
            if (BF16)
                reinterpret_cast<__nv_bfloat16*>(wout)[e] = __float2bfloat16_rn(w);
            else
                reinterpret_cast<float*>(wout)[e] = w;
        }
    }
}

__global__ void k_init_state(BuildView b, float* __restrict__ V, float* __restrict__ c,
                             uint8_t* __restrict__ ref) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.Npad) return;
    float v = 0.0f;
    if (i < b.N) {
        const U4 u = philox4x32_10(i, 0u, TAG_INIT, 0u, b.key0, b.key1);
        v = __fmul_rn(b.V_th, unit24(u.x));
    }
    V[i] = v;
    c[i] = 0.0f;
    ref[i] = 0;
}

cudaError_t launch_build_cdf(const BuildView& b, cudaStream_t s) {
    k_build_cdf<<<b.n_modules, 256, 0, s>>>(b);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_gen_synapses(const BuildView& b, uint32_t* td, void* w, cudaStream_t s) {
    const uint64_t threads = (uint64_t)b.N * (b.Kpad >> 2);
    if (threads == 0) return cudaSuccess;
    const uint64_t blocks = (threads + 255) / 256;
    if (b.w_bf16)
        k_gen_synapses<true><<<(unsigned)blocks, 256, 0, s>>>(b, td, w);
    else
        k_gen_synapses<false><<<(unsigned)blocks, 256, 0, s>>>(b, td, w);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_gen_grouped(const BuildView& b, uint32_t* td, void* w, cudaStream_t s) {
    if (b.N == 0 || b.Kpad == 0) return cudaSuccess;
    const int warps = 8;
    const size_t smem = (size_t)warps * (b.max_off + 1) * sizeof(uint32_t);
    const void* fn = b.w_bf16 ? (const void*)k_gen_grouped<true> : (const void*)k_gen_grouped<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (b.N + warps - 1) / warps;
    if (b.w_bf16)
        k_gen_grouped<true><<<blocks, warps * 32, smem, s>>>(b, td, w);
    else
        k_gen_grouped<false><<<blocks, warps * 32, smem, s>>>(b, td, w);
    count_launch(1);
    return cudaGetLastError();
}

static unsigned pair_blocks(const BuildView& b) {
    return (unsigned)(((uint64_t)b.N * b.pair_n + 255) / 256);
}

cudaError_t launch_pair_count(const BuildView& b, cudaStream_t s) {
    if (b.N == 0 || b.pair_n == 0) return cudaSuccess;
    k_pair_count<<<pair_blocks(b), 256, 0, s>>>(b);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pair_rows(const BuildView& b, cudaStream_t s) {
    if (b.N == 0) return cudaSuccess;
    k_pair_rows<<<(b.N + 7) / 8, 256, 0, s>>>(b);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pair_fill(const BuildView& b, uint32_t* td, void* w, cudaStream_t s) {
    if (b.N == 0 || b.pair_n == 0) return cudaSuccess;
    k_pair_fill<<<pair_blocks(b), 256, 0, s>>>(b, td);
    const uint64_t threads = (uint64_t)b.N * (b.Kpad >> 2);
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (threads) {
        if (b.w_bf16)
            k_pair_attr<true><<<blocks, 256, 0, s>>>(b, td, w);
        else
            k_pair_attr<false><<<blocks, 256, 0, s>>>(b, td, w);
    }
    count_launch(threads ? 2 : 1);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const BuildView& b, float* V, float* c, uint8_t* ref, cudaStream_t s) {
    k_init_state<<<(b.Npad + 255) / 256, 256, 0, s>>>(b, V, c, ref);
    count_launch(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spatial decomposition (Sec. II-D, deferred arborization of Sec. II-C): the
// target-side copy of a shard.  For the sources [h0, h0 + rows) whose stencil
// reaches the shard's neurons [n0, n1), the synapses of their rows (the fixed
// out-degree law, drawn exactly as k_gen_synapses draws them) that target the
// shard, in draw order: one warp per source row.  Pass 1 counts them.
__global__ void __launch_bounds__(256) k_shard_count(BuildView b, uint32_t h0, uint32_t rows, uint32_t n0, uint32_t n1,
                                                     uint32_t* __restrict__ cnt) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;  // warp-uniform
    const uint32_t i = h0 + r;
    const uint32_t s = i / b.M;
    const bool exc = (i - s * b.M) < b.n_exc;
    const uint32_t* T = b.cdf_T + (size_t)s * b.max_off;
    const uint32_t* TM = b.cdf_mod + (size_t)s * b.max_off;
    const uint32_t n = __ldg(b.cdf_n + s);
    uint32_t c = 0;
    for (uint32_t k = lane; k < b.K; k += 32) {
        const Draw d = draw_synapse(b, i, k, exc, T, TM, n);
        c += (d.tgt >= n0 && d.tgt < n1) ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) cnt[r] = c;
}

// Pass 2: the kept synapses of row r at [row_ptr[r], row_ptr[r + 1]): target
// neuron - n0 | delay << 24 and the weight.
template <bool BF16>
__global__ void __launch_bounds__(256) k_shard_fill(BuildView b, uint32_t h0, uint32_t rows, uint32_t n0, uint32_t n1,
                                                    const uint64_t* __restrict__ row_ptr, uint32_t* __restrict__ td,
                                                    void* __restrict__ wout) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;  // warp-uniform
    const uint32_t i = h0 + r;
    const uint32_t s = i / b.M;
    const bool exc = (i - s * b.M) < b.n_exc;
    const uint32_t* T = b.cdf_T + (size_t)s * b.max_off;
    const uint32_t* TM = b.cdf_mod + (size_t)s * b.max_off;
    const uint32_t n = __ldg(b.cdf_n + s);
    uint64_t pos = row_ptr[r];
    for (uint32_t k0 = 0; k0 < b.K; k0 += 32) {
        const uint32_t k = k0 + lane;
        Draw d{0u, 0u, 0u, 0.0f};
        bool keep = false;
        if (k < b.K) {
            d = draw_synapse(b, i, k, exc, T, TM, n);
            keep = d.tgt >= n0 && d.tgt < n1;
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, keep);
        if (keep) {
            const uint64_t e = pos + __popc(m & ((1u << lane) - 1u));
            td[e] = (d.tgt - n0) | (d.d << 24);
            if (BF16)
                reinterpret_cast<__nv_bfloat16*>(wout)[e] = __float2bfloat16_rn(d.w);
            else
                reinterpret_cast<float*>(wout)[e] = d.w;
        }
        pos += __popc(m);
    }
}

// V = V_th U[0,1), c = 0, ref = 0 for the neurons [n0, n0 + count) of a shard
// (the draw of k_init_state, by global neuron id).
__global__ void k_shard_init(BuildView b, uint32_t n0, uint32_t count, float* __restrict__ V, float* __restrict__ c,
                             uint8_t* __restrict__ ref) {
    const uint32_t li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= count) return;
    const U4 u = philox4x32_10(n0 + li, 0u, TAG_INIT, 0u, b.key0, b.key1);
    V[li] = __fmul_rn(b.V_th, unit24(u.x));
    c[li] = 0.0f;
    ref[li] = 0;
}

cudaError_t launch_shard_count(const BuildView& b, uint32_t h0, uint32_t rows, uint32_t n0, uint32_t n1, uint32_t* cnt,
                               cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    k_shard_count<<<(rows + 7) / 8, 256, 0, s>>>(b, h0, rows, n0, n1, cnt);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_shard_fill(const BuildView& b, uint32_t h0, uint32_t rows, uint32_t n0, uint32_t n1,
                              const uint64_t* row_ptr, uint32_t* td, void* w, cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    if (b.w_bf16)
        k_shard_fill<true><<<(rows + 7) / 8, 256, 0, s>>>(b, h0, rows, n0, n1, row_ptr, td, w);
    else
        k_shard_fill<false><<<(rows + 7) / 8, 256, 0, s>>>(b, h0, rows, n0, n1, row_ptr, td, w);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_shard_init(const BuildView& b, uint32_t n0, uint32_t count, float* V, float* c, uint8_t* ref,
                              cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_shard_init<<<(count + 255) / 256, 256, 0, s>>>(b, n0, count, V, c, ref);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace snn
