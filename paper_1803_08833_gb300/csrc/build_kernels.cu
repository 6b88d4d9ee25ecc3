// build_kernels.cu -- construction phase (Sec. II-A phase 1, Sec. II-B, Sec. III-B).
//
//   k_build_cdf    per source module: FP64 lateral-kernel values over the in-grid
//                  modules of the cut-off disc, their normalisation (the A / B
//                  constants of Sec. I and Sec. III-B) and cumulative distribution,
//                  converted to uint32 thresholds.
//   k_gen_synapses per (neuron, 4 synapses): Philox draws -> target module by
//                  inverse CDF, target neuron, weight, delay; 16 B vector stores.
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

template <bool BF16>
__global__ void __launch_bounds__(256) k_gen_synapses(BuildView b, uint32_t* __restrict__ tgt,
                                                      void* __restrict__ wout, uint8_t* __restrict__ dout) {
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
            if (exc) {
                w[q] = __fadd_rn(b.w_lo, __fmul_rn(b.w_span, unit24(u.z)));
                d[q] = b.d_lo + __umulhi(u.w, b.d_span);
            } else {
                w[q] = b.w_inh;
                d[q] = b.d_inh;
            }
        }
    }
    const size_t e = (size_t)i * b.Kpad + k0;
    *reinterpret_cast<uint4*>(tgt + e) = make_uint4(tg[0], tg[1], tg[2], tg[3]);
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
    *reinterpret_cast<uint32_t*>(dout + e) = d[0] | (d[1] << 8) | (d[2] << 16) | (d[3] << 24);
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

cudaError_t launch_gen_synapses(const BuildView& b, uint32_t* tgt, void* w, uint8_t* d, cudaStream_t s) {
    const uint64_t threads = (uint64_t)b.N * (b.Kpad >> 2);
    if (threads == 0) return cudaSuccess;
    const uint64_t blocks = (threads + 255) / 256;
    if (b.w_bf16)
        k_gen_synapses<true><<<(unsigned)blocks, 256, 0, s>>>(b, tgt, w, d);
    else
        k_gen_synapses<false><<<(unsigned)blocks, 256, 0, s>>>(b, tgt, w, d);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const BuildView& b, float* V, float* c, uint8_t* ref, cudaStream_t s) {
    k_init_state<<<(b.Npad + 255) / 256, 256, 0, s>>>(b, V, c, ref);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace snn
