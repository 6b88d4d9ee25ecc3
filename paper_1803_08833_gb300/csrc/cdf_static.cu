// cdf_static.cu -- target-module tables built without any device allocation.
//
// Some callers cannot let this library allocate device memory: a process whose
// device memory is owned by a pool or arena (a serving framework, an embedded
// runtime) must not have it fragmented or over-committed behind its back, and
// a latency-critical loop cannot afford the implicit device-wide
// synchronisation of cudaMalloc/cudaFree.  snn_build_cdf_static builds the
// same tables as snn_build_network into buffers the caller already owns; the
// only extra device memory it uses is the fixed scratch below, which is part
// of the loaded library image.
#include "snn.h"
#include "snn_internal.h"

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

namespace {

// Fixed scratch: per (source module, stencil offset) FP64 kernel values and
// their running sums; the stencil offsets themselves.  Every GPU that loads
// the library holds both arrays (4 MiB + 16 KiB) until the process exits.
constexpr size_t kMaxScratchDoubles = (size_t)1 << 19;  // modules x stencil offsets
constexpr size_t kMaxOffsets = 4096;                     // stencil offsets (dx, dy pairs)

static __device__ __align__(256) double g_cdf_scratch[kMaxScratchDoubles];
static __device__ __align__(256) int16_t g_cdf_offsets[2 * kMaxOffsets];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};
int16_t* g_offsets_ptr[kMaxDevices] = {};

// The in-disc offsets (dx, dy) with dx^2 + dy^2 <= R2 in (dy, dx) raster
// order, at most n entries (the host's count of the same rule).
__global__ void k_disc_offsets(int R, uint32_t R2, uint32_t n, int16_t* out) {
    uint32_t k = 0;
    for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx)
            if ((uint32_t)(dx * dx + dy * dy) <= R2 && k < n) {
                out[2 * k] = (int16_t)dx;
                out[2 * k + 1] = (int16_t)dy;
                ++k;
            }
}

snn_status static_fail(snn_status s, const std::string& msg) {
    snn::set_last_error(msg.c_str());
    return s;
}

// Device addresses of the fixed arrays on the current device.  The host-side
// names are only stand-ins for the device symbols, so the addresses must come
// from cudaGetSymbolAddress, once per device, with that device current.
snn_status device_addresses(double** scratch, int16_t** offsets) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(SNN_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(SNN_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cdf_scratch);
        if (e != cudaSuccess)
            return static_fail(SNN_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        void* q = nullptr;
        e = cudaGetSymbolAddress(&q, g_cdf_offsets);
        if (e != cudaSuccess)
            return static_fail(SNN_ECUDA, std::string("cudaGetSymbolAddress(offsets): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = (double*)p;
        g_offsets_ptr[dev] = (int16_t*)q;
    }
    *scratch = g_scratch_ptr[dev];
    *offsets = g_offsets_ptr[dev];
    return SNN_OK;
}

}  // namespace

extern "C" {

snn_status snn_build_cdf_static(const snn_config* cfg, uint32_t* thresh, uint32_t* tgt_module, uint32_t* counts,
                                uint32_t* max_offsets, void* stream) {
    if (!cfg) return static_fail(SNN_EINVAL, "config is NULL");
    if (cfg->grid_w == 0 || cfg->grid_h == 0) return static_fail(SNN_EINVAL, "grid_w and grid_h must be positive");
    if (!(cfg->spacing_um > 0.0f)) return static_fail(SNN_EINVAL, "spacing_um must be positive");
    if (cfg->kernel != SNN_KERNEL_GAUSS && cfg->kernel != SNN_KERNEL_EXP)
        return static_fail(SNN_EINVAL, "kernel must be SNN_KERNEL_GAUSS or SNN_KERNEL_EXP");
    if ((cfg->kernel == SNN_KERNEL_GAUSS && !(cfg->sigma_um > 0.0)) ||
        (cfg->kernel == SNN_KERNEL_EXP && !(cfg->lambda_um > 0.0)))
        return static_fail(SNN_EINVAL, "kernel length scale must be positive");
    if (!(cfg->cutoff_um >= 0.0) || cfg->cutoff_um / cfg->spacing_um > 512.0)
        return static_fail(SNN_EINVAL, "cutoff_um must be in [0, 512 * spacing_um]");

    // the stencil: in-disc offsets in (dy, dx) raster order (counted on the
    // host by the same rule snn_build_network uses; written on the device)
    uint32_t R2 = 0;
    const std::vector<int16_t> off = snn::disc_offsets(*cfg, &R2);
    int R = 0;
    while ((uint32_t)((R + 1) * (R + 1)) <= R2) ++R;
    const uint32_t n_off = (uint32_t)(off.size() / 2);
    const uint64_t n_modules = (uint64_t)cfg->grid_w * cfg->grid_h;
    if (max_offsets) *max_offsets = n_off;
    if (!thresh && !tgt_module && !counts) return SNN_OK;  // size query
    if (!thresh || !tgt_module || !counts) return static_fail(SNN_EINVAL, "thresh, tgt_module and counts must all be set");
    if (n_off > kMaxOffsets) {
        char buf[160];
        snprintf(buf, sizeof buf, "stencil of %u offsets exceeds the fixed limit of %zu", n_off, kMaxOffsets);
        return static_fail(SNN_EINVAL, buf);
    }
    if (n_modules * n_off > kMaxScratchDoubles) {
        char buf[200];
        snprintf(buf, sizeof buf, "modules x stencil offsets = %llu exceeds the fixed scratch of %zu entries",
                 (unsigned long long)(n_modules * n_off), kMaxScratchDoubles);
        return static_fail(SNN_EINVAL, buf);
    }

    double* scratch = nullptr;
    int16_t* doff = nullptr;
    snn_status st = device_addresses(&scratch, &doff);
    if (st != SNN_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    // The offsets are a pure function of the cut-off: a one-thread kernel writes
    // them into the fixed array (no host-to-device copy, so every work item of
    // the call is a kernel on `stream`).
    k_disc_offsets<<<1, 1, 0, s>>>(R, R2, n_off, doff);
    snn::count_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(SNN_ECUDA, std::string("k_disc_offsets: ") + cudaGetErrorString(e));

    // The scratch needs no clearing: the kernel writes every entry it reads.
    snn::BuildView b{};
    b.grid_w = cfg->grid_w;
    b.grid_h = cfg->grid_h;
    b.n_modules = (uint32_t)n_modules;
    b.max_off = n_off;
    b.kernel = cfg->kernel;
    b.spacing = (double)cfg->spacing_um;
    b.sigma = cfg->sigma_um;
    b.lambda = cfg->lambda_um;
    b.offsets = doff;
    b.scratch = scratch;
    b.cdf_T = thresh;
    b.cdf_mod = tgt_module;
    b.cdf_n = counts;
    e = snn::launch_build_cdf(b, s);
    if (e != cudaSuccess) return static_fail(SNN_ECUDA, std::string("k_build_cdf: ") + cudaGetErrorString(e));
    return SNN_OK;
}

}  // extern "C"
