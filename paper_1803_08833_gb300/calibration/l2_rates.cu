// l2_rates.cu -- memory-system rates that bound spike delivery on this GPU.
//
// Measures, with CUDA events: (1) random 4-byte red.global.add.s32 into
// buffers of several sizes (the delay ring takes one such reduction per
// synaptic event), (2) the same with the 32 lanes of a warp on consecutive
// words, (3) a streaming 16-byte read of a 4 GB table (the synapse table
// stream), (4) the stream with one random reduction per loaded word, (5)
// reads of short contiguous segments at random places of a region of the
// table (segment length x region size: the access pattern of a delivery
// that reads a few dozen synapses per row), (6) random reductions whose
// addresses are restricted to one value of a single address bit chosen per
// CTA from its SM index (four ways of halving the SMs, bits 7-24): the largest
// rate difference between the two halves, to look for a die-local placement.
// Prints one JSON object.  Every address is inside its buffer.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

__global__ void k_red_random(int* buf, uint32_t n, uint32_t R, uint32_t salt) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t r = 0; r < R; ++r) {
        const uint32_t a = mix32(g * 977u + r * 131071u + salt) % n;
        asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(buf + a), "r"(1) : "memory");
    }
}

__global__ void k_red_coalesced(int* buf, uint32_t n, uint32_t R, uint32_t salt) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31, w = g >> 5;
    for (uint32_t r = 0; r < R; ++r) {
        const uint32_t a = (mix32(w * 977u + r * 131071u + salt) % (n / 32)) * 32 + lane;
        asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(buf + a), "r"(1) : "memory");
    }
}

__global__ void k_stream(const uint4* tab, size_t n16, uint32_t* sink) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint4 v = __ldcs(tab + i);
        acc += v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x12345678u) sink[0] = acc;
}

__global__ void k_stream_red(const uint4* tab, size_t n16, int* buf, uint32_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint4 v = __ldcs(tab + i);
        const uint32_t t[4] = {v.x % n, v.y % n, v.z % n, v.w % n};
        for (int q = 0; q < 4; ++q)
            asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(buf + t[q]), "r"(1) : "memory");
    }
}

// Each warp reads `segs` segments of CH x 128 bytes at random 128-byte aligned
// offsets of the first `region` bytes, 8 segments in flight.  The chunk count
// is a template constant so that every load of a round is issued before the
// first is used (a runtime-bounded inner loop kept the loaded words in local
// memory and serialised the reads).
template <int CH>
__global__ void k_seg_read(const uint32_t* tab, size_t region, uint32_t segs, uint32_t salt, uint32_t* sink) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t slots = (region - CH * 128) / 128;
    uint32_t acc = 0;
    for (uint32_t s0 = 0; s0 < segs; s0 += 8) {
        uint32_t v[8][CH];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const size_t base =
                ((size_t)mix32(w * 7919u + (s0 + u) * 104729u + salt) * 2654435761ull % slots) * 32;  // words
#pragma unroll
            for (int k = 0; k < CH; ++k) v[u][k] = __ldcs(tab + base + k * 32 + lane);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < CH; ++k) acc ^= v[u][k];
    }
    if (acc == 0x12345678u) sink[0] = acc;
}

__device__ __forceinline__ uint32_t sm_index() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Random reductions into nwords words whose byte-address bit b equals
// group(smid) ^ flip; the address is built inside the buffer.
__global__ void k_red_halves(int* buf, uint32_t nwords, uint32_t b, uint32_t mode, uint32_t flip, uint32_t R,
                             uint32_t salt) {
    const uint32_t sm = sm_index();
    uint32_t g;
    if (mode == 0)
        g = sm < 76 ? 0u : 1u;
    else if (mode == 1)
        g = sm & 1u;
    else if (mode == 2)
        g = (sm >> 1) & 1u;
    else
        g = (sm / 38) & 1u;
    const uint32_t bit = g ^ flip, wb = b - 2, half = nwords >> 1;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t r = 0; r < R; ++r) {
        const uint32_t a = mix32(t * 977u + r * 131071u + salt) % half;
        const uint32_t w = ((a >> wb) << (wb + 1)) | (bit << wb) | (a & ((1u << wb) - 1u));
        asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(buf + w), "r"(1) : "memory");
    }
}

__global__ void k_fill(uint4* tab, size_t n16) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
        tab[i] = make_uint4(mix32((uint32_t)i * 4), mix32((uint32_t)i * 4 + 1), mix32((uint32_t)i * 4 + 2),
                            mix32((uint32_t)i * 4 + 3));
}

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const uint32_t sizes_mb[] = {4, 16, 60, 256, 1024};
    const uint32_t max_words = 1024u << 18;  // 1 GiB of int32
    int* buf = nullptr;
    uint4* tab = nullptr;
    uint32_t* sink = nullptr;
    const size_t tab_bytes = (size_t)4 << 30;
    if (cudaMalloc(&buf, (size_t)max_words * 4) != cudaSuccess || cudaMalloc(&tab, tab_bytes) != cudaSuccess ||
        cudaMalloc(&sink, 64) != cudaSuccess) {
        printf("{\"error\": \"allocation failed\"}\n");
        return 1;
    }
    cudaMemset(buf, 0, (size_t)max_words * 4);
    k_fill<<<sms * 8, 256>>>(tab, tab_bytes / 16);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.0f;
    const int grid = sms * 16;
    const uint32_t R = 32;
    const double total = (double)grid * 256 * R;
    printf("{\"sms\": %d, \"random_red_per_s\": {", sms);
    for (int k = 0; k < 5; ++k) {
        const uint32_t n = sizes_mb[k] << 18;
        k_red_random<<<grid, 256>>>(buf, n, R, 1);
        cudaEventRecord(a);
        for (int it = 0; it < 5; ++it) k_red_random<<<grid, 256>>>(buf, n, R, 7 + it);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        printf("%s\"%u MB\": %.4g", k ? ", " : "", sizes_mb[k], 5.0 * total / (ms * 1e-3));
    }
    printf("}, \"coalesced_red_per_s\": {");
    for (int k = 0; k < 5; ++k) {
        const uint32_t n = sizes_mb[k] << 18;
        cudaEventRecord(a);
        for (int it = 0; it < 5; ++it) k_red_coalesced<<<grid, 256>>>(buf, n, R, 7 + it);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        printf("%s\"%u MB\": %.4g", k ? ", " : "", sizes_mb[k], 5.0 * total / (ms * 1e-3));
    }
    cudaEventRecord(a);
    for (int it = 0; it < 3; ++it) k_stream<<<sms * 8, 256>>>(tab, tab_bytes / 16, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    printf("}, \"stream_read_gb_per_s\": %.1f", 3.0 * tab_bytes / (ms * 1e-3) / 1e9);
    const size_t part = tab_bytes / 16 / 16;
    const uint32_t n60 = 60u << 18;
    cudaEventRecord(a);
    k_stream_red<<<sms * 16, 256>>>(tab, part, buf, n60);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    printf(", \"stream_plus_random_red\": {\"red_per_s\": %.4g, \"table_gb_per_s\": %.1f}", part * 4.0 / (ms * 1e-3),
           part * 16.0 / (ms * 1e-3) / 1e9);
    // short segments at random places: 128 B, 512 B and 1 KB over 512 MB, 1 GB and 4 GB
    printf(", \"segment_read_gb_per_s\": {");
    const size_t regions[] = {(size_t)512 << 20, (size_t)1 << 30, tab_bytes};
    const uint32_t lens[] = {128, 512, 1024};
    const uint32_t segs = 64;
    int first = 1;
    for (uint32_t L : lens)
        for (size_t R : regions) {
            const int sgrid = sms * 8;
            const double bytes = (double)sgrid * 8 * segs * L;  // 8 warps per block
            auto seg = [&](uint32_t salt) {
                if (L == 128) k_seg_read<1><<<sgrid, 256>>>((const uint32_t*)tab, R, segs, salt, sink);
                if (L == 512) k_seg_read<4><<<sgrid, 256>>>((const uint32_t*)tab, R, segs, salt, sink);
                if (L == 1024) k_seg_read<8><<<sgrid, 256>>>((const uint32_t*)tab, R, segs, salt, sink);
            };
            seg(3);
            cudaEventRecord(a);
            for (int it = 0; it < 3; ++it) seg(11 + it);
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&ms, a, b);
            printf("%s\"%u B in %zu MB\": %.1f", first ? "" : ", ", L, R >> 20, 3.0 * bytes / (ms * 1e-3) / 1e9);
            first = 0;
        }
    printf("}");
    // reductions by SM half and address bit (16 M words = 64 MB of the reduction buffer)
    {
        const uint32_t nw = 16u << 20;
        const int hgrid = sms * 8;
        const double hr = (double)hgrid * 256 * 64;
        double worst = 0.0, lo = 1e300, hi = 0.0;
        for (uint32_t mode = 0; mode < 4; ++mode)
            for (uint32_t bb = 7; bb <= 24; ++bb) {
                double r2[2];
                for (uint32_t flip = 0; flip < 2; ++flip) {
                    k_red_halves<<<hgrid, 256>>>(buf, nw, bb, mode, flip, 64, 1);
                    cudaEventRecord(a);
                    for (int it = 0; it < 3; ++it) k_red_halves<<<hgrid, 256>>>(buf, nw, bb, mode, flip, 64, 3 + it);
                    cudaEventRecord(b);
                    cudaEventSynchronize(b);
                    cudaEventElapsedTime(&ms, a, b);
                    r2[flip] = 3.0 * hr / (ms * 1e-3);
                    lo = r2[flip] < lo ? r2[flip] : lo;
                    hi = r2[flip] > hi ? r2[flip] : hi;
                }
                const double d = (r2[0] > r2[1] ? r2[0] - r2[1] : r2[1] - r2[0]) / (0.5 * (r2[0] + r2[1]));
                worst = d > worst ? d : worst;
            }
        printf(", \"red_by_sm_half_and_address_bit\": {\"max_rel_difference\": %.4f, \"min_per_s\": %.4g, "
               "\"max_per_s\": %.4g}", worst, lo, hi);
    }
    const cudaError_t e = cudaGetLastError();
    printf(", \"status\": \"%s\"}\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
