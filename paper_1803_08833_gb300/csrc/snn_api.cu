// snn_api.cu -- host runtime and C ABI of libsnn.so (declared in include/snn.h).
//
// The host side validates the network description, derives the constants of
// the method once in FP64 (membrane and fatigue decay factors of Eq. 1-2, the
// Poisson table of the external synapses, fixed-point scales), obtains device
// memory from the caller's allocator, and enqueues the kernels.  Nothing of
// the simulation itself runs on the host.
#include "snn.h"
#include "snn_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace snn;

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

snn_status fail(snn_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
snn_status fail(snn_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define CUDA_TRY(expr)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(SNN_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                           \
    } while (0)

constexpr int TIMING_SLOTS = 256;

struct EventRing {
    cudaEvent_t a[TIMING_SLOTS] = {};
    cudaEvent_t b[TIMING_SLOTS] = {};
    bool pending[TIMING_SLOTS] = {};
    uint64_t next = 0;
    double total_ms = 0.0;
    uint64_t count = 0;
};

}  // namespace

namespace snn {
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace snn

struct snn_net {
    snn_config cfg;
    snn_alloc_fn alloc_fn = nullptr;
    snn_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;
    std::vector<void*> blocks;
    uint64_t device_bytes = 0;
    int device = 0;

    uint32_t N = 0, Npad = 0, M = 0, K = 0, Kpad = 0, n_modules = 0, n_exc = 0, D = 0;
    uint32_t max_off = 0, nb = 0;
    NetView v{};
    uint32_t* cdf_T = nullptr;
    uint32_t* cdf_mod = nullptr;
    uint32_t* cdf_n = nullptr;

    int schedule = 0;
    int block = 256;
    int grid = 0;       // delivery grid of schedules 0 and 1
    int pgrid = 0;      // persistent grid (schedule 2)
    int tgrid = 0;      // tiled persistent grid (schedule 3), 0 if unavailable
    int ogrid = 0;      // owner-windowed persistent grid (schedule 4), 0 until set up
    int plgrid = 0;     // pulled windowed persistent grid (schedule 5), 0 until set up
    size_t pull_runs_bytes = 0;
    int pull_mode = 0;  // schedule 5 bands in use: 1 uniform, 2 module-aligned
    bool stdp = false;        // spike-timing dependent plasticity (schedules 0 and 1)
    StdpView sp{};
    int2* own_rec = nullptr;  // schedule 4 record queues and their size
    size_t own_rec_bytes = 0;
    uint32_t pair_n = 0;              // pairwise law: stencil entries
    uint2* band_ids_dev = nullptr;    // banded delivery tables
    uint32_t* band_rng_dev = nullptr;
    int timing_every = 0;
    uint64_t step_calls = 0;
    EventRing ev_deliver, ev_neuron, ev_persist;
};

namespace {

void* dev_alloc(snn_net* n, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (n->alloc_fn) {
        p = n->alloc_fn(bytes, n->alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        n->blocks.push_back(p);
        n->device_bytes += bytes;
    }
    return p;
}

void release_all(snn_net* n) {
    for (void* p : n->blocks) {
        if (n->free_fn)
            n->free_fn(p, n->alloc_ctx);
        else if (!n->alloc_fn)
            cudaFree(p);
    }
    n->blocks.clear();
}

void destroy_events(EventRing& r) {
    for (int i = 0; i < TIMING_SLOTS; ++i) {
        if (r.a[i]) cudaEventDestroy(r.a[i]);
        if (r.b[i]) cudaEventDestroy(r.b[i]);
        r.a[i] = r.b[i] = nullptr;
    }
}

snn_status validate(const snn_config* c) {
    if (!c) return fail(SNN_EINVAL, "config is NULL");
    if (c->grid_w == 0 || c->grid_h == 0 || c->neurons_per_module == 0)
        return fail(SNN_EINVAL, "grid_w, grid_h and neurons_per_module must be positive");
    const uint64_t N = (uint64_t)c->grid_w * c->grid_h * c->neurons_per_module;
    if (N > (uint64_t)MAX_NEURON_BLOCKS * NEURONS_PER_BLOCK)
        return fail(SNN_EINVAL, "too many neurons (%llu > %u)", (unsigned long long)N,
                    MAX_NEURON_BLOCKS * NEURONS_PER_BLOCK);
    if (c->conn_rule != SNN_RULE_FIXED_K && c->conn_rule != SNN_RULE_PAIRWISE)
        return fail(SNN_EINVAL, "conn_rule must be SNN_RULE_FIXED_K or SNN_RULE_PAIRWISE");
    if (c->conn_rule == SNN_RULE_FIXED_K && c->K > 16384) return fail(SNN_EINVAL, "K must be <= 16384");
    if (c->conn_rule == SNN_RULE_PAIRWISE) {
        if (!(c->p_local >= 0.0f && c->p_local <= 1.0f) || !(c->A_remote >= 0.0 && c->A_remote <= 1.0) ||
            !(c->p_min > 0.0 && c->p_min < 1.0))
            return fail(SNN_EINVAL, "pairwise rule: need 0 <= p_local <= 1, 0 <= A_remote <= 1, 0 < p_min < 1");
        if (c->neurons_per_module > MAX_ROW)
            return fail(SNN_EINVAL, "pairwise rule: neurons_per_module must be <= %u", MAX_ROW);
        if (c->table_layout != SNN_LAYOUT_DRAW)
            return fail(SNN_EINVAL, "pairwise rule: rows come in stencil order; table_layout must be SNN_LAYOUT_DRAW");
    }
    if ((c->weight_dist != SNN_WDIST_UNIFORM && c->weight_dist != SNN_WDIST_GAUSS) || !(c->w_exc_sd >= 0.0f) ||
        !(c->w_inh_sd >= 0.0f) || !std::isfinite(c->w_exc_sd) || !std::isfinite(c->w_inh_sd))
        return fail(SNN_EINVAL, "weight_dist must be SNN_WDIST_UNIFORM or SNN_WDIST_GAUSS with finite sd >= 0");
    if ((c->delay_dist != SNN_DDIST_UNIFORM && c->delay_dist != SNN_DDIST_EXP) ||
        (c->delay_dist == SNN_DDIST_EXP && !(c->delay_tau_ms > 0.0f && std::isfinite(c->delay_tau_ms))))
        return fail(SNN_EINVAL, "delay_dist must be SNN_DDIST_UNIFORM, or SNN_DDIST_EXP with delay_tau_ms > 0");
    if (!(c->exc_fraction >= 0.0f && c->exc_fraction <= 1.0f))
        return fail(SNN_EINVAL, "exc_fraction must be in [0, 1]");
    if (!(c->spacing_um > 0.0f)) return fail(SNN_EINVAL, "spacing_um must be positive");
    if (c->kernel != SNN_KERNEL_GAUSS && c->kernel != SNN_KERNEL_EXP)
        return fail(SNN_EINVAL, "kernel must be SNN_KERNEL_GAUSS or SNN_KERNEL_EXP");
    if (c->kernel == SNN_KERNEL_GAUSS && !(c->sigma_um > 0.0))
        return fail(SNN_EINVAL, "sigma_um must be positive");
    if (c->kernel == SNN_KERNEL_EXP && !(c->lambda_um > 0.0))
        return fail(SNN_EINVAL, "lambda_um must be positive");
    if (!(c->cutoff_um >= 0.0) || c->cutoff_um / c->spacing_um > 512.0)
        return fail(SNN_EINVAL, "cutoff_um must be in [0, 512 * spacing_um]");
    if (c->d_exc_lo < 1 || c->d_exc_hi < c->d_exc_lo || c->d_exc_hi > 255 || c->d_inh < 1 ||
        c->d_inh > 255)
        return fail(SNN_EINVAL, "delays must satisfy 1 <= d_exc_lo <= d_exc_hi <= 255, 1 <= d_inh <= 255");
    if (!(c->tau_m_ms > 0.0f) || !(c->tau_c_ms > 0.0f) || !(c->dt_ms > 0.0f))
        return fail(SNN_EINVAL, "tau_m_ms, tau_c_ms and dt_ms must be positive");
    if (!(c->t_ref_ms >= 0.0f) || std::lround((double)c->t_ref_ms / c->dt_ms) > 255)
        return fail(SNN_EINVAL, "t_ref_ms must be in [0, 255 dt]");
    if (!(c->ext_rate_hz >= 0.0f)) return fail(SNN_EINVAL, "ext_rate_hz must be >= 0");
    if (!(c->imposed_rate_hz >= 0.0f)) return fail(SNN_EINVAL, "imposed_rate_hz must be >= 0");
    if (c->weight_dtype != SNN_WEIGHT_F32 && c->weight_dtype != SNN_WEIGHT_BF16)
        return fail(SNN_EINVAL, "weight_dtype must be SNN_WEIGHT_F32 or SNN_WEIGHT_BF16");
    if (c->fx_shift < 8 || c->fx_shift > 24) return fail(SNN_EINVAL, "fx_shift must be in [8, 24]");
    if (c->stdp != 0 && c->stdp != 1) return fail(SNN_EINVAL, "stdp must be 0 or 1");
    if (c->stdp &&
        (!(c->stdp_tau_plus_ms > 0.0f) || !(c->stdp_tau_minus_ms > 0.0f) || !(c->stdp_w_max >= 0.0f) ||
         !std::isfinite(c->stdp_A_plus) || !std::isfinite(c->stdp_A_minus) || !std::isfinite(c->stdp_w_max) ||
         c->stdp_period_steps == 0 || c->weight_dtype != SNN_WEIGHT_F32))
        return fail(SNN_EINVAL, "stdp needs tau_plus, tau_minus > 0, finite amplitudes, w_max >= 0, a period "
                                ">= 1 and f32 weights");
    if (c->table_layout != SNN_LAYOUT_DRAW && c->table_layout != SNN_LAYOUT_GROUPED)
        return fail(SNN_EINVAL, "table_layout must be SNN_LAYOUT_DRAW or SNN_LAYOUT_GROUPED");
    if (!std::isfinite(c->w_exc_lo) || !std::isfinite(c->w_exc_hi) || !std::isfinite(c->w_inh) ||
        !std::isfinite(c->V_th_mV) || !std::isfinite(c->V_reset_mV) || !std::isfinite(c->E_mV) ||
        !std::isfinite(c->J_ext_mV) || !std::isfinite(c->g_c_mV) || !std::isfinite(c->alpha_c))
        return fail(SNN_EINVAL, "non-finite parameter");
    float wmax = std::fmax(std::fabs(c->w_exc_lo), std::fmax(std::fabs(c->w_exc_hi), std::fabs(c->w_inh)));
    if (c->weight_dist == SNN_WDIST_GAUSS)  // the table's extreme quantiles lie within 4 sd of the mean
        wmax = std::fmax(std::fabs(0.5f * (c->w_exc_lo + c->w_exc_hi)) + 4.0f * c->w_exc_sd,
                         std::fabs(c->w_inh) + 4.0f * c->w_inh_sd);
    if (std::ldexp((double)wmax, (int)c->fx_shift) > 1.0e9 ||
        std::ldexp((double)std::fabs(c->J_ext_mV), (int)c->fx_shift) > 1.0e8)
        return fail(SNN_EINVAL, "weights too large for the fixed-point scale");
    return SNN_OK;
}

// Host-side constants of the method (FP64, rounded once to float).
snn_status derive(snn_net* n) {
    const snn_config& c = n->cfg;
    n->M = c.neurons_per_module;
    n->N = c.grid_w * c.grid_h * c.neurons_per_module;
    n->nb = (n->N + NEURONS_PER_BLOCK - 1) / NEURONS_PER_BLOCK;
    if (n->nb == 0) n->nb = 1;
    n->Npad = n->nb * NEURONS_PER_BLOCK;
    n->K = c.K;
    n->Kpad = (c.K + K_ALIGN - 1) / K_ALIGN * K_ALIGN;
    n->n_modules = c.grid_w * c.grid_h;
    double ne = std::floor((double)c.exc_fraction * (double)c.neurons_per_module + 0.5);
    if (ne > (double)c.neurons_per_module) ne = (double)c.neurons_per_module;
    n->n_exc = (uint32_t)ne;
    n->D = (c.d_exc_hi > c.d_inh ? c.d_exc_hi : c.d_inh) + 1u;

    NetView& v = n->v;
    v.N = n->N;
    v.Npad = n->Npad;
    v.M = n->M;
    v.K = n->K;
    v.Kpad = n->Kpad;
    v.n_exc = n->n_exc;
    v.D = n->D;
    v.nb = n->nb;
    v.key0 = (uint32_t)c.seed;
    v.key1 = (uint32_t)(c.seed >> 32);
    v.ref_steps = (uint32_t)std::lround((double)c.t_ref_ms / (double)c.dt_ms);

    const double dt = c.dt_ms, tau_m = c.tau_m_ms, tau_c = c.tau_c_ms;
    const double decay_m = std::exp(-dt / tau_m);
    const double decay_c = std::exp(-dt / tau_c);
    // Eq. 1 driven by c(s) = c0 exp(-s/tau_c): the adaptation term integrated
    // over one step contributes -k_c c0, k_c = g_c int_0^dt exp(-(dt-s)/tau_m) exp(-s/tau_c) ds.
    const double kc = (tau_c == tau_m) ? (double)c.g_c_mV * dt * decay_m
                                       : (double)c.g_c_mV * (tau_m * tau_c / (tau_c - tau_m)) * (decay_c - decay_m);
    v.a_m = (float)decay_m;
    v.a_c = (float)decay_c;
    v.kc = (float)kc;
    v.E = c.E_mV;
    v.V_th = c.V_th_mV;
    v.V_reset = c.V_reset_mV;
    v.alpha_c = c.alpha_c;
    v.w_scale = std::ldexp(1.0f, (int)c.fx_shift);
    v.in_scale = std::ldexp(1.0f, -(int)c.fx_shift);
    v.J_ext_fx = (int32_t)std::lrintf(c.J_ext_mV * v.w_scale);
    v.w_bf16 = c.weight_dtype == SNN_WEIGHT_BF16 ? 1 : 0;

    // External Poisson synapses: P[k] = floor(F(k) 2^32), F the Poisson CDF of
    // mean rate * dt; the count of a step is #{k : P[k] <= u} for a uniform
    // 32-bit u.  The table stops before the first entry that reaches 2^32 - 1.
    const double mean = (double)c.ext_rate_hz * dt / 1000.0;
    v.pois_len = 0;
    if (mean > 0.0) {
        double pmf = std::exp(-mean), F = 0.0;
        for (uint32_t k = 0;; ++k) {
            F = F + pmf;
            const double x = std::floor(F * 4294967296.0);
            if (x >= 4294967295.0) break;
            if (k >= (uint32_t)MAX_POIS) return fail(SNN_EINVAL, "ext_rate_hz * dt too large for the Poisson table");
            v.pois32[v.pois_len++] = (uint32_t)x;
            pmf = pmf * mean / (double)(k + 1);
        }
    }
    v.pois_pad = 0;
    if (v.pois_len) {
        v.pois_pad = 1;
        while (v.pois_pad < v.pois_len) v.pois_pad <<= 1;
    }
    for (uint32_t k = v.pois_len; k < (uint32_t)MAX_POIS; ++k) v.pois32[k] = 0xFFFFFFFFu;
    double pf = (double)c.imposed_rate_hz * dt / 1000.0;
    if (pf > 1.0) pf = 1.0;
    v.imposed_thresh = (uint64_t)std::floor(pf * 4294967296.0);
    v.raster_cap = c.raster_capacity;
    v.wait_limit_ns = 2000000000ull;
    v.barrier_extra = 0;
    return SNN_OK;
}

}  // namespace

namespace snn {
// In-disc grid offsets (dx, dy) with dx^2 + dy^2 <= R2, in (dy, dx) raster order.
std::vector<int16_t> disc_offsets(const snn_config& c, uint32_t* R2_out) {
    const double q = c.cutoff_um / (double)c.spacing_um;
    const uint32_t R2 = (uint32_t)std::floor(q * q + 1e-9);
    int R = 0;
    while ((uint32_t)((R + 1) * (R + 1)) <= R2) ++R;
    std::vector<int16_t> off;
    for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx)
            if ((uint32_t)(dx * dx + dy * dy) <= R2) {
                off.push_back((int16_t)dx);
                off.push_back((int16_t)dy);
            }
    *R2_out = R2;
    return off;
}
}  // namespace snn

namespace {

// Unnormalised lateral shape f at squared grid distance d2 (the same
// expression order as the device kernel of the target-module tables).
double lateral_shape(const snn_config& c, uint32_t d2) {
    const double sp = (double)c.spacing_um;
    if (c.kernel == SNN_KERNEL_GAUSS) {
        const double num = (double)d2 * sp * sp;
        const double den = 2.0 * c.sigma_um * c.sigma_um;
        return std::exp(-(num / den));
    }
    const double r = sp * std::sqrt((double)d2);
    return std::exp(-(r / c.lambda_um));
}

// Standard normal quantile: the rational approximation of P. J. Acklam (2003)
// refined by two Halley steps on the CDF 0.5 erfc(-x / sqrt 2).
double normal_quantile(double p) {
    static const double a[6] = {-3.969683028665376e+01, 2.209460984245205e+02, -2.759285104469687e+02,
                                1.383577518672690e+02,  -3.066479806614716e+01, 2.506628277459239e+00};
    static const double b[5] = {-5.447609879822406e+01, 1.615858368580409e+02, -1.556989798598866e+02,
                                6.680131188771972e+01,  -1.328068155288572e+01};
    static const double c[6] = {-7.784894002430293e-03, -3.223964580411365e-01, -2.400758277161838e+00,
                                -2.549732539343734e+00, 4.374664141464968e+00,  2.938163982698783e+00};
    static const double d[4] = {7.784695709041462e-03, 3.224671290700398e-01, 2.445134137142996e+00,
                                3.754408661907416e+00};
    const double plow = 0.02425;
    double x;
    if (p < plow) {
        const double q = std::sqrt(-2.0 * std::log(p));
        x = (((((c[0] * q + c[1]) * q + c[2]) * q + c[3]) * q + c[4]) * q + c[5]) /
            ((((d[0] * q + d[1]) * q + d[2]) * q + d[3]) * q + 1.0);
    } else if (p > 1.0 - plow) {
        const double q = std::sqrt(-2.0 * std::log(1.0 - p));
        x = -(((((c[0] * q + c[1]) * q + c[2]) * q + c[3]) * q + c[4]) * q + c[5]) /
            ((((d[0] * q + d[1]) * q + d[2]) * q + d[3]) * q + 1.0);
    } else {
        const double q = p - 0.5, r = q * q;
        x = (((((a[0] * r + a[1]) * r + a[2]) * r + a[3]) * r + a[4]) * r + a[5]) * q /
            (((((b[0] * r + b[1]) * r + b[2]) * r + b[3]) * r + b[4]) * r + 1.0);
    }
    for (int it = 0; it < 2; ++it) {
        const double e = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
        const double u = e * std::sqrt(2.0 * 3.14159265358979323846) * std::exp(0.5 * x * x);
        x = x - u / (1.0 + 0.5 * x * u);
    }
    return x;
}

// Construction tables derived on the host in FP64.
struct HostTables {
    std::vector<int32_t> pdx, pdy;  // pairwise stencil, (dy, dx) order
    std::vector<uint64_t> pthr;     // floor(p 2^32), 2^32 = always
    std::vector<float> wtab;        // 2 x WTAB Gaussian efficacy quantiles (excitatory, inhibitory)
    std::vector<uint64_t> dthr;     // exponential delay thresholds
};

void host_tables(const snn_config& c, HostTables* t) {
    if (c.conn_rule == SNN_RULE_PAIRWISE) {
        // stencil radius: grow while the pair probability on an axis exceeds p_min
        uint32_t R = 0;
        while (R < 4096 && c.A_remote * lateral_shape(c, (R + 1) * (R + 1)) > c.p_min) ++R;
        for (int y = -(int)R; y <= (int)R; ++y)
            for (int x = -(int)R; x <= (int)R; ++x) {
                double p;
                if (x == 0 && y == 0) {
                    p = (double)c.p_local;
                } else {
                    p = c.A_remote * lateral_shape(c, (uint32_t)(x * x + y * y));
                    if (!(p > c.p_min)) continue;
                }
                t->pdx.push_back(x);
                t->pdy.push_back(y);
                t->pthr.push_back(p >= 1.0 ? 4294967296ull : (uint64_t)std::floor(p * 4294967296.0));
            }
    }
    if (c.weight_dist == SNN_WDIST_GAUSS) {
        t->wtab.resize(2 * WTAB);
        for (int pop = 0; pop < 2; ++pop) {
            const double mean = pop == 0 ? 0.5 * ((double)c.w_exc_lo + (double)c.w_exc_hi) : (double)c.w_inh;
            const double sd = pop == 0 ? (double)c.w_exc_sd : (double)c.w_inh_sd;
            for (uint32_t k = 0; k < WTAB; ++k) {
                double w = mean + sd * normal_quantile(((double)k + 0.5) / (double)WTAB);
                if (pop == 0 && w < 0.0) w = 0.0;  // efficacies keep the sign of their population
                if (pop == 1 && w > 0.0) w = 0.0;
                t->wtab[pop * WTAB + k] = (float)w;
            }
        }
    }
    if (c.delay_dist == SNN_DDIST_EXP) {
        // P(delay <= d_lo + k) = (1 - e^{-(k+1)/tau}) / (1 - e^{-span/tau}), tau in steps
        const uint32_t span = c.d_exc_hi - c.d_exc_lo + 1u;
        const double tau = (double)c.delay_tau_ms / (double)c.dt_ms;
        const double Z = 1.0 - std::exp(-(double)span / tau);
        for (uint32_t k = 0; k + 1 < span; ++k) {
            const double F = (1.0 - std::exp(-(double)(k + 1) / tau)) / Z;
            const double x = std::floor(F * 4294967296.0);
            t->dthr.push_back(x >= 4294967296.0 ? 4294967296ull : (uint64_t)x);
        }
    }
}

}  // namespace

namespace snn {
// Bounds used by memory estimates: the longest row of the pairwise rule (mean
// of an interior excitatory neuron plus eight standard deviations) and its
// stencil size.
void pairwise_bounds(const snn_config& c, uint32_t* max_row, uint32_t* stencil) {
    HostTables t;
    host_tables(c, &t);
    double mean = 0.0;
    for (size_t k = 0; k < t.pthr.size(); ++k) mean += (double)t.pthr[k] / 4294967296.0 * c.neurons_per_module;
    *max_row = (uint32_t)std::ceil(mean + 8.0 * std::sqrt(mean) + 16.0);
    *stencil = (uint32_t)t.pthr.size();
}
}  // namespace snn

namespace {

void free_block(snn_net* n, void* p, size_t bytes) {
    for (size_t i = 0; i < n->blocks.size(); ++i)
        if (n->blocks[i] == p) {
            if (n->free_fn)
                n->free_fn(p, n->alloc_ctx);
            else if (!n->alloc_fn)
                cudaFree(p);
            n->blocks.erase(n->blocks.begin() + i);
            n->device_bytes -= (bytes + 255) & ~(size_t)255;
            return;
        }
}

// Owner-windowed delivery (schedule 4): bands of ceil(Q / G) quads, one per
// CTA of a grid of one CTA per SM; a window of `window` steps (0 = the largest
// that fits in shared memory, at most D - 1); record queues of `queue_cap`
// entries per (owner, producer) (0 = twice the expected near events of a step
// at the larger of the imposed rate and 10 Hz, plus 64, in [64, 4096]).
snn_status owned_setup(snn_net* n, uint32_t window, uint32_t queue_cap) {
    NetView& v = n->v;
    const int G = owned_grid();
    if (G <= 0) return fail(SNN_ECUDA, "schedule 4: no multiprocessor count");
    const uint32_t Q = n->Npad / 4;
    const uint32_t BQ = (Q + (uint32_t)G - 1) / (uint32_t)G;
    const uint32_t Wmax = owned_max_window(v, G, BQ);
    if (Wmax == 0)
        return fail(SNN_EINVAL, "schedule 4: a delay window row of %u neurons per CTA does not fit in shared memory",
                    BQ * 4);
    const uint32_t W = window == 0 ? Wmax : window;
    if (W > Wmax) return fail(SNN_EINVAL, "schedule 4: window %u exceeds the %u steps that fit (D - 1 = %u)", W, Wmax,
                              v.D - 1);
    uint32_t cap = queue_cap;
    if (cap == 0) {
        const double rate = std::max(10.0, (double)n->cfg.imposed_rate_hz);
        const double ev = (double)n->N * n->K * rate * n->cfg.dt_ms / 1000.0;
        cap = (uint32_t)std::min(4096.0, std::max(64.0, 2.0 * ev / ((double)G * G) + 64.0));
        cap = (cap + 31) / 32 * 32;
    }
    if (cap > (1u << 20)) return fail(SNN_EINVAL, "schedule 4: queue capacity %u exceeds 2^20", cap);
    const uint64_t magic = ((uint64_t)1 << 32) / BQ + (((uint64_t)1 << 32) % BQ ? 1 : 0);
    for (uint32_t q = 0; q < Q; ++q) {  // the band arithmetic of the kernel, checked for every quad
        uint32_t b = (uint32_t)(((uint64_t)q * magic) >> 32);
        if ((uint64_t)b * BQ > q) --b;
        if (!((uint64_t)b * BQ <= q && q < (uint64_t)(b + 1) * BQ))
            return fail(SNN_EINVAL, "schedule 4: band arithmetic fails for quad %u", q);
    }
    const size_t rec_bytes = (size_t)G * G * cap * sizeof(int2);
    if (!n->own_rec || rec_bytes != n->own_rec_bytes || n->ogrid != G) {
        if (n->own_rec) free_block(n, n->own_rec, n->own_rec_bytes);
        n->own_rec = (int2*)dev_alloc(n, rec_bytes);
        if (!n->own_rec) return fail(SNN_ENOMEM, "schedule 4: device allocation of %zu bytes of queues failed", rec_bytes);
        n->own_rec_bytes = rec_bytes;
    }
    if (!v.own_cnt || n->ogrid != G) {
        v.own_cnt = (uint32_t*)dev_alloc(n, (size_t)G * G * 4);
        v.own_ovf = (uint32_t*)dev_alloc(n, (size_t)G * 4);
        if (!v.own_cnt || !v.own_ovf) return fail(SNN_ENOMEM, "schedule 4: device allocation of queue counters failed");
        CUDA_TRY(cudaMemset(v.own_ovf, 0, (size_t)G * 4));
        CUDA_TRY(cudaMemset(v.own_cnt, 0, (size_t)G * G * 4));
    }
    v.own_rec = n->own_rec;
    v.own_W = W;
    v.own_BQ = BQ;
    v.own_cap = cap;
    v.own_magic = magic;
    n->ogrid = G;
    return SNN_OK;
}

// Pulled windowed delivery (schedule 5): one band of quads per CTA of a grid
// of one CTA per SM, each with its table of runs (source module, stencil
// entries of the band's target modules); a window of `window` steps (0 = the
// largest that fits in shared memory, at most D - 1).  band_mode 1: bands of
// ceil(Q / G) quads; 2: bands on module boundaries (a band then reads only
// synapses it owns, but bands differ in size by up to u modules); 0: 2 if its
// largest band is at most a uniform band plus one module (the synapses a
// uniform band reads beyond its own) and fits in shared memory, else 1.  Needs
// the grouped layout (rows ordered by target module) with K synapses per row.
// The stencil the rows' segment index follows, as (dx, dy) pairs in its order,
// and whether every offset numbers an entry (per-pair law) or only the in-grid
// ones (fixed out-degree law).
std::vector<int16_t> pull_stencil(const snn_config& c, bool* all_entries) {
    std::vector<int16_t> off;
    if (c.conn_rule == SNN_RULE_PAIRWISE) {
        HostTables ht;
        host_tables(c, &ht);
        for (size_t k = 0; k < ht.pdx.size(); ++k) {
            off.push_back((int16_t)ht.pdx[k]);
            off.push_back((int16_t)ht.pdy[k]);
        }
        *all_entries = true;
    } else {
        uint32_t R2 = 0;
        off = disc_offsets(c, &R2);
        *all_entries = false;
    }
    return off;
}

snn_status pull_setup(snn_net* n, uint32_t window, int32_t band_mode) {
    NetView& v = n->v;
    const bool pairwise = n->cfg.conn_rule == SNN_RULE_PAIRWISE;
    if (!v.segidx || (!pairwise && (n->cfg.table_layout != SNN_LAYOUT_GROUPED || v.row_len)))
        return fail(SNN_EINVAL, "schedule 5 needs rows grouped by target module: table_layout = "
                                "SNN_LAYOUT_GROUPED, or the per-pair law");
    if (n->K > pull_k_max()) return fail(SNN_EINVAL, "schedule 5: K = %u exceeds %u", n->K, pull_k_max());
    if (band_mode < 0 || band_mode > 2) return fail(SNN_EINVAL, "schedule 5: band_mode must be 0, 1 or 2");
    const int G = owned_grid();
    if (G <= 0) return fail(SNN_ECUDA, "schedule 5: no multiprocessor count");
    const uint32_t Q = n->Npad / 4;
    bool all_entries = false;
    const std::vector<int16_t> off = pull_stencil(n->cfg, &all_entries);
    struct Plan {
        std::vector<uint32_t> bq, ptr;
        std::vector<uint2> runs;
        uint32_t BQ = 0, R_max = 0, Wmax = 0;
    } plan[2];
    for (int k = 0; k < 2; ++k) {
        if (band_mode != 0 && band_mode != k + 1) continue;
        Plan& p = plan[k];
        p.bq = pull_bands(n->N, n->M, Q, (uint32_t)G, k == 1);
        for (int b = 0; b < G; ++b) p.BQ = std::max(p.BQ, p.bq[b + 1] - p.bq[b]);
        p.R_max = pull_build_runs(n->N, n->M, n->cfg.grid_w, n->cfg.grid_h, off, p.bq, p.runs, p.ptr, all_entries);
        p.Wmax = p.BQ ? pull_max_window(v, G, p.BQ, p.R_max) : 0;
    }
    int pick = band_mode == 2 ? 1 : 0;
    if (band_mode == 0 && plan[1].Wmax > 0 && (uint64_t)plan[1].BQ * 4 <= (uint64_t)plan[0].BQ * 4 + n->M) pick = 1;
    Plan& p = plan[pick];
    const uint32_t BQ = p.BQ, R_max = p.R_max, Wmax = p.Wmax;
    std::vector<uint2>& runs = p.runs;
    std::vector<uint32_t>& ptr = p.ptr;
    for (const uint2& r : runs)  // the kernel's reads of the segment index stay in the row
        if ((r.y & 0xFFFFu) >= (r.y >> 16) || (r.y >> 16) >= v.seg_stride || r.x >= n->n_modules)
            return fail(SNN_EINVAL, "schedule 5: run table entry out of range");
    if (Wmax == 0)
        return fail(SNN_EINVAL, "schedule 5: a delay window row of %u neurons per CTA does not fit in shared memory",
                    BQ * 4);
    const uint32_t W = window == 0 ? Wmax : window;
    if (W > Wmax) return fail(SNN_EINVAL, "schedule 5: window %u exceeds the %u steps that fit (D - 1 = %u)", W, Wmax,
                              v.D - 1);
    uint32_t tchunks = 0;
    const uint32_t tcols = pull_tmem_cols(BQ, &tchunks);
    if (tcols == 0)
        return fail(SNN_EINVAL, "schedule 5: the state of a band of %u neurons does not fit in tensor memory", BQ * 4);
    cudaStream_t s = 0;
    if (n->plgrid != G || !v.pull_seg) {
        const size_t warps = (size_t)G * pull_warps();
        struct Req {
            void** p;
            size_t bytes;
        } reqs[] = {
            {(void**)&v.pull_seg, (size_t)n->Npad * 2 * 4},
            {(void**)&v.pull_segmod, (size_t)n->Npad * 2 * 4},
            {(void**)&v.pull_mcnt, (size_t)n->n_modules * 3 * 4},
            {(void**)&v.pull_woff, warps * 2 * 4},
            {(void**)&v.pull_run_ptr, (size_t)(G + 1) * 4},
            {(void**)&v.pull_bq, (size_t)(G + 1) * 4},
        };
        for (auto& r : reqs) {
            *r.p = dev_alloc(n, r.bytes);
            if (!*r.p) return fail(SNN_ENOMEM, "schedule 5: device allocation of %zu bytes failed", r.bytes);
        }
        CUDA_TRY(cudaMemsetAsync(v.pull_seg, 0, (size_t)n->Npad * 2 * 4, s));
        CUDA_TRY(cudaMemsetAsync(v.pull_segmod, 0, (size_t)n->Npad * 2 * 4, s));
    }
    if (v.pull_runs) free_block(n, (void*)v.pull_runs, n->pull_runs_bytes);
    v.pull_runs = nullptr;
    n->pull_runs_bytes = std::max<size_t>(runs.size(), 1) * sizeof(uint2);
    uint2* druns = (uint2*)dev_alloc(n, n->pull_runs_bytes);
    if (!druns) return fail(SNN_ENOMEM, "schedule 5: device allocation of the run table failed");
    if (!runs.empty())
        CUDA_TRY(cudaMemcpyAsync(druns, runs.data(), runs.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync((void*)v.pull_run_ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync((void*)v.pull_bq, p.bq.data(), p.bq.size() * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
    v.pull_runs = druns;
    v.pull_W = W;
    v.pull_BQ = BQ;
    v.pull_R_max = R_max;
    v.pull_tmem_chunks = tchunks;
    v.pull_tmem_cols = tcols;
    v.pull_aligned = 0;
    if (pick == 1) {  // every module in one band: counted by its owner when no band holds too many
        uint32_t most = 0;
        for (int b = 0; b < G; ++b)
            if (p.bq[b + 1] > p.bq[b])
                most = std::max(most, (std::min(p.bq[b + 1] * 4, n->N) - 1) / n->M - p.bq[b] * 4 / n->M + 1);
        v.pull_aligned = most <= pull_mods_max() ? 1u : 0u;
    }
    n->plgrid = G;
    n->pull_mode = pick + 1;
    return SNN_OK;
}

// Bands of target module rows for the persistent delivery.  bands = 0 picks
// ceil(ring bytes / (L2 / 2)), at most grid_h / (2 R + 1) for a stencil of
// row radius R (1 when the ring fits).  Measured on GB300 (events/s): the
// 242 MB ring of the 48x48 grid 3 bands 7.2e10, 4 bands 8.1e10, 6 bands
// 7.7e10 (the per-pair 48x48: 9.4e10 / 9.5e10 / 8.9e10); the 968 MB ring of
// the 96x96 grid 12 bands 6.4-6.6e10, 13 6.2e10, 15 6.1e10, 20 5.6e10: per-band
// ring columns must fit in about half the L2, but bands lower than the
// stencil split every spiking row into more short pieces.  Needs a segment
// index (grouped layout, or the pairwise law, whose rows are grouped by
// construction).
snn_status set_bands(snn_net* n, uint32_t bands, uint32_t* chosen) {
    const snn_config& c = n->cfg;
    NetView& v = n->v;
    const bool pairwise = c.conn_rule == SNN_RULE_PAIRWISE;
    // stencil rows (dy) in segment-index order
    std::vector<int> sdx, sdy;
    if (v.segidx && (bands == 0 || bands > 1)) {
        if (pairwise) {
            HostTables ht;
            host_tables(c, &ht);
            sdx.assign(ht.pdx.begin(), ht.pdx.end());
            sdy.assign(ht.pdy.begin(), ht.pdy.end());
        } else {
            uint32_t R2 = 0;
            std::vector<int16_t> off = disc_offsets(c, &R2);
            for (size_t o = 0; o < off.size(); o += 2) {
                sdx.push_back(off[o]);
                sdy.push_back(off[o + 1]);
            }
        }
    }
    int R = 0;
    for (int dy : sdy) R = std::max(R, std::abs(dy));
    if (bands == 0) {
        int dev = 0, l2 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        const double ring = (double)n->D * n->Npad * 4.0;
        const double budget = l2 > 0 ? 0.5 * l2 : 32.0 * (1 << 20);
        bands = v.segidx ? (uint32_t)std::ceil(ring / budget) : 1u;
        bands = std::min<uint32_t>(bands, std::max<uint32_t>(1u, c.grid_h / (2 * (uint32_t)R + 1)));
        bands = std::min<uint32_t>(std::max<uint32_t>(bands, 1u), c.grid_h);
    }
    if (bands < 1 || bands > c.grid_h) return fail(SNN_EINVAL, "bands must be in [1, grid_h = %u]", c.grid_h);
    if (bands > 1 && !v.segidx)
        return fail(SNN_EINVAL, "banded delivery needs a segment index: table_layout = SNN_LAYOUT_GROUPED or the "
                                "pairwise law");
    if (chosen) *chosen = bands;
    v.n_bands = bands;
    if (bands == 1) return SNN_OK;
    if (sdy.size() + 1 > 0xFFFFu) return fail(SNN_EINVAL, "stencil too large for banded delivery");
    const uint32_t H = c.grid_h, W = c.grid_w, M = c.neurons_per_module;
    std::vector<uint32_t> row(bands + 1);
    for (uint32_t b = 0; b <= bands; ++b) row[b] = (uint32_t)((uint64_t)H * b / bands);
    std::vector<uint2> ids(bands);
    for (uint32_t b = 0; b < bands; ++b) {
        const int lo = std::max(0, (int)row[b] - R), hi = std::min((int)H, (int)row[b + 1] + R);
        ids[b] = make_uint2((uint32_t)lo * W * M, (uint32_t)hi * W * M);
    }
    const uint32_t keys = pairwise ? H : n->n_modules;
    std::vector<uint32_t> rng((size_t)keys * bands);
    for (uint32_t k = 0; k < keys; ++k) {
        const int sx = pairwise ? 0 : (int)(k % W), sy = pairwise ? (int)k : (int)(k / W);
        // target rows of the entries, in segment-index order (all entries of the
        // pairwise stencil; the in-grid entries of the fixed law's table)
        std::vector<int> ty;
        for (size_t o = 0; o < sdy.size(); ++o) {
            const int tx = sx + sdx[o], y = sy + sdy[o];
            if (!pairwise && (tx < 0 || y < 0 || tx >= (int)W || y >= (int)H)) continue;
            ty.push_back(y);
        }
        for (uint32_t b = 0; b < bands; ++b) {
            uint32_t j0 = 0, j1 = 0;
            for (int y : ty) {
                j0 += y < (int)row[b] ? 1u : 0u;
                j1 += y < (int)row[b + 1] ? 1u : 0u;
            }
            rng[(size_t)k * bands + b] = j0 | (j1 << 16);
        }
    }
    if (!n->band_ids_dev) {  // room for the largest band count
        n->band_ids_dev = (uint2*)dev_alloc(n, (size_t)H * sizeof(uint2));
        n->band_rng_dev = (uint32_t*)dev_alloc(n, (size_t)keys * H * 4);
        if (!n->band_ids_dev || !n->band_rng_dev) return fail(SNN_ENOMEM, "device allocation of the band tables failed");
    }
    CUDA_TRY(cudaMemcpy(n->band_ids_dev, ids.data(), ids.size() * sizeof(uint2), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(n->band_rng_dev, rng.data(), rng.size() * 4, cudaMemcpyHostToDevice));
    v.band_key_row = pairwise ? 1u : 0u;
    v.band_ids = n->band_ids_dev;
    v.band_rng = n->band_rng_dev;
    return SNN_OK;
}

// Plasticity state of a freshly built table: traces, histories and
// accumulators at zero, decays from the time constants (FP64, rounded once),
// and the incoming index (synapses of every target), counted, scanned on the
// host and filled.
snn_status stdp_setup(snn_net* n, cudaStream_t s) {
    const snn_config& c = n->cfg;
    const NetView& v = n->v;
    StdpView& p = n->sp;
    const size_t Np = n->Npad, D = n->D;
    const size_t nsyn = (size_t)n->N * n->Kpad;
    p.y = (float*)dev_alloc(n, Np * 4);
    p.x = (float*)dev_alloc(n, Np * 4);
    p.xh = (float*)dev_alloc(n, (D + 1) * Np * 4);
    p.hist = (uint32_t*)dev_alloc(n, D * Np * 4);
    p.hist_cnt = (uint32_t*)dev_alloc(n, D * 4);
    p.delta = (int32_t*)dev_alloc(n, nsyn * 4);
    uint64_t* in_ptr = (uint64_t*)dev_alloc(n, ((size_t)n->N + 1) * 8);
    uint64_t* cursor = (uint64_t*)dev_alloc(n, ((size_t)n->N + 1) * 8);
    if (!p.y || !p.x || !p.xh || !p.hist || !p.hist_cnt || !p.delta || !in_ptr || !cursor)
        return fail(SNN_ENOMEM, "device allocation of the plasticity state failed");
    CUDA_TRY(cudaMemsetAsync(p.y, 0, Np * 4, s));
    CUDA_TRY(cudaMemsetAsync(p.x, 0, Np * 4, s));
    CUDA_TRY(cudaMemsetAsync(p.xh, 0, (D + 1) * Np * 4, s));
    CUDA_TRY(cudaMemsetAsync(p.hist_cnt, 0, D * 4, s));
    CUDA_TRY(cudaMemsetAsync(p.delta, 0, nsyn * 4, s));
    CUDA_TRY(cudaMemsetAsync(cursor, 0, ((size_t)n->N + 1) * 8, s));
    CUDA_TRY(launch_stdp_index(v, cursor, nullptr, s));  // counts per target
    std::vector<uint64_t> h((size_t)n->N + 1, 0);
    CUDA_TRY(cudaMemcpyAsync(h.data(), cursor, (size_t)n->N * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    uint64_t acc = 0;
    for (size_t j = 0; j <= n->N; ++j) {
        const uint64_t x = j < n->N ? h[j] : 0;
        h[j] = acc;
        acc += x;
    }
    uint64_t* in_syn = (uint64_t*)dev_alloc(n, std::max<uint64_t>(acc, 1) * 8);
    if (!in_syn) return fail(SNN_ENOMEM, "device allocation of the incoming-synapse index failed");
    CUDA_TRY(cudaMemcpyAsync(in_ptr, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(cursor, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(launch_stdp_index(v, cursor, in_syn, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // the host vector goes out of scope
    p.in_ptr = in_ptr;
    p.in_syn = in_syn;
    p.a_plus = (float)std::exp(-(double)c.dt_ms / (double)c.stdp_tau_plus_ms);
    p.a_minus = (float)std::exp(-(double)c.dt_ms / (double)c.stdp_tau_minus_ms);
    p.A_plus = c.stdp_A_plus;
    p.A_minus = c.stdp_A_minus;
    p.w_max = c.stdp_w_max;
    p.period = c.stdp_period_steps;
    n->stdp = true;
    return SNN_OK;
}

// The scalar parameters of the construction kernels (device tables are set
// by the caller); n->max_off must be set.
void fill_build_view(const snn_net* n, BuildView& b) {
    const snn_config& c = n->cfg;
    const NetView& v = n->v;
    b.grid_w = c.grid_w;
    b.grid_h = c.grid_h;
    b.n_modules = n->n_modules;
    b.max_off = n->max_off;
    b.M = n->M;
    b.N = n->N;
    b.Npad = n->Npad;
    b.n_exc = n->n_exc;
    b.d_lo = c.d_exc_lo;
    b.d_span = c.d_exc_hi - c.d_exc_lo + 1u;
    b.d_inh = c.d_inh;
    b.key0 = v.key0;
    b.key1 = v.key1;
    b.kernel = c.kernel;
    b.spacing = (double)c.spacing_um;
    b.sigma = c.sigma_um;
    b.lambda = c.lambda_um;
    b.w_lo = c.w_exc_lo;
    b.w_span = c.w_exc_hi - c.w_exc_lo;
    b.w_inh = c.w_inh;
    b.V_th = c.V_th_mV;
    b.w_bf16 = v.w_bf16;
    b.weight_dist = c.weight_dist;
    b.delay_dist = c.delay_dist;
    b.inh_local_only = c.inh_local_only;
}

snn_status build_impl(snn_net* n, cudaStream_t s) {
    const snn_config& c = n->cfg;
    snn_status st = derive(n);
    if (st != SNN_OK) return st;
    uint32_t R2 = 0;
    std::vector<int16_t> off = disc_offsets(c, &R2);
    n->max_off = (uint32_t)(off.size() / 2);

    NetView& v = n->v;
    n->pgrid = persistent_grid(v.w_bf16 != 0);
    const bool pairwise = c.conn_rule == SNN_RULE_PAIRWISE;
    HostTables ht;
    host_tables(c, &ht);

    BuildView b{};
    fill_build_view(n, b);

    // construction-only buffers, released at the end of the build
    std::vector<std::pair<void*, size_t>> temps;
    auto temp = [&](size_t bytes) -> void* {
        void* p = dev_alloc(n, bytes);
        if (p) temps.push_back({p, bytes});
        return p;
    };
    if (!ht.wtab.empty()) {
        float* wt = (float*)temp(ht.wtab.size() * 4);
        if (!wt) return fail(SNN_ENOMEM, "device allocation of the efficacy table failed");
        CUDA_TRY(cudaMemcpyAsync(wt, ht.wtab.data(), ht.wtab.size() * 4, cudaMemcpyHostToDevice, s));
        b.wtab = wt;
    }
    if (!ht.dthr.empty()) {
        uint64_t* dt = (uint64_t*)temp(ht.dthr.size() * 8);
        if (!dt) return fail(SNN_ENOMEM, "device allocation of the delay table failed");
        CUDA_TRY(cudaMemcpyAsync(dt, ht.dthr.data(), ht.dthr.size() * 8, cudaMemcpyHostToDevice, s));
        b.dthr = dt;
        b.n_dthr = (uint32_t)ht.dthr.size();
    }
    if (pairwise) {
        // out-degrees first: the row stride of the table is the longest row
        b.pair_n = (uint32_t)ht.pdx.size();
        int32_t* pdx = (int32_t*)temp(ht.pdx.size() * 4);
        int32_t* pdy = (int32_t*)temp(ht.pdy.size() * 4);
        uint64_t* pthr = (uint64_t*)temp(ht.pthr.size() * 8);
        // per (neuron, stencil entry) counts, then the rows' segment index (kept)
        uint16_t* pcnt = (uint16_t*)dev_alloc(n, (size_t)n->N * (b.pair_n + 1) * 2);
        uint32_t* maxl = (uint32_t*)temp(4);
        uint32_t* rlen = (uint32_t*)dev_alloc(n, (size_t)n->N * 4);
        if (!pdx || !pdy || !pthr || !pcnt || !maxl || !rlen)
            return fail(SNN_ENOMEM, "device allocation of the pairwise construction buffers failed");
        CUDA_TRY(cudaMemcpyAsync(pdx, ht.pdx.data(), ht.pdx.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(pdy, ht.pdy.data(), ht.pdy.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(pthr, ht.pthr.data(), ht.pthr.size() * 8, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemsetAsync(maxl, 0, 4, s));
        b.pair_dx = pdx;
        b.pair_dy = pdy;
        b.pair_thr = pthr;
        b.pair_cnt = pcnt;
        b.row_len = rlen;
        b.max_len = maxl;
        CUDA_TRY(launch_pair_count(b, s));
        CUDA_TRY(launch_pair_rows(b, s));
        uint32_t longest = 0;
        CUDA_TRY(cudaMemcpyAsync(&longest, maxl, 4, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (longest > MAX_ROW) return fail(SNN_EINVAL, "pairwise rule: a row of %u synapses exceeds %u", longest, MAX_ROW);
        n->K = longest;
        n->Kpad = (longest + K_ALIGN - 1) / K_ALIGN * K_ALIGN;
        v.K = n->K;
        v.Kpad = n->Kpad;
        v.row_len = rlen;
        n->pair_n = b.pair_n;
    }
    b.K = n->K;
    b.Kpad = n->Kpad;
    const size_t nsyn = (size_t)n->N * n->Kpad;
    // the persistent kernels' per-CTA arrays hold any of their grids: at most 8 CTAs per SM
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, n->device);
    const size_t persist_bound = (size_t)8 * (sms > 0 ? sms : 1) > (size_t)n->pgrid ? (size_t)8 * (sms > 0 ? sms : 1)
                                                                                    : (size_t)n->pgrid;
    const size_t wbytes = v.w_bf16 ? 2 : 4;
    struct Req {
        void** p;
        size_t bytes;
    } reqs[] = {
        {(void**)&v.td, nsyn * 4},
        {(void**)&v.w, nsyn * wbytes},
        {(void**)&v.V, (size_t)n->Npad * 4},
        {(void**)&v.c, (size_t)n->Npad * 4},
        {(void**)&v.ref, (size_t)n->Npad},
        {(void**)&v.ring, (size_t)n->D * n->Npad * 4},
        {(void**)&v.seg, (size_t)n->Npad * 4},
        {(void**)&v.blk_cnt, (size_t)n->nb * 4},
        {(void**)&v.blk_off, (size_t)(n->nb + 1) * 4},
        {(void**)&v.blk_ext, (size_t)n->nb * 8},
        {(void**)&v.blk_rec, (size_t)n->nb * 8},
        {(void**)&v.raster_t, (size_t)(c.raster_capacity ? c.raster_capacity : 1) * 4},
        {(void**)&v.raster_id, (size_t)(c.raster_capacity ? c.raster_capacity : 1) * 4},
        {(void**)&v.st, sizeof(DevState)},
        {(void**)&v.woff, persist_bound * 32 * 4},  // per-warp counts: any persistent grid, <= 32 warps per CTA
        {(void**)&v.cta_cnt, persist_bound * 4},
        {(void**)&v.cta_speed, persist_bound * 4},
        {(void**)&n->cdf_T, (size_t)n->n_modules * n->max_off * 4},
        {(void**)&n->cdf_mod, (size_t)n->n_modules * n->max_off * 4},
        {(void**)&n->cdf_n, (size_t)n->n_modules * 4},
        {(void**)&v.mod_cnt, (size_t)n->n_modules * 2 * 4},
        {(void**)&v.seg_mod, (size_t)n->Npad * 4},
    };
    for (auto& r : reqs) {
        *r.p = dev_alloc(n, r.bytes);
        if (!*r.p) return fail(SNN_ENOMEM, "device allocation of %zu bytes failed", r.bytes);
    }
    const bool grouped = c.table_layout == SNN_LAYOUT_GROUPED;
    uint16_t* segidx = nullptr;
    v.n_modules = n->n_modules;
    v.max_off = n->max_off;
    v.seg_stride = n->max_off + 1;
    v.grid_w = c.grid_w;
    v.n_bands = 1;
    if (pairwise) {  // the pairwise rows are grouped by construction
        v.segidx = b.pair_cnt;
        v.seg_stride = b.pair_n + 1;
    }
    if (grouped) {
        // per-row segment index and, per target module, its incoming (source, stencil index) list
        segidx = (uint16_t*)dev_alloc(n, (size_t)n->N * v.seg_stride * sizeof(uint16_t));
        uint32_t* in_src = (uint32_t*)dev_alloc(n, (size_t)n->n_modules * n->max_off * 4);
        uint32_t* in_j = (uint32_t*)dev_alloc(n, (size_t)n->n_modules * n->max_off * 4);
        uint32_t* in_cnt = (uint32_t*)dev_alloc(n, (size_t)n->n_modules * 4);
        if (!segidx || !in_src || !in_j || !in_cnt) return fail(SNN_ENOMEM, "device allocation of the segment index failed");
        std::vector<uint32_t> h_src((size_t)n->n_modules * n->max_off, 0), h_j(h_src.size(), 0), h_cnt(n->n_modules, 0);
        for (uint32_t sm = 0; sm < n->n_modules; ++sm) {
            const int sx = (int)(sm % c.grid_w), sy = (int)(sm / c.grid_w);
            uint32_t j = 0;
            for (size_t o = 0; o < off.size(); o += 2) {
                const int tx = sx + off[o], ty = sy + off[o + 1];
                if (tx < 0 || ty < 0 || tx >= (int)c.grid_w || ty >= (int)c.grid_h) continue;
                const uint32_t tm = (uint32_t)ty * c.grid_w + (uint32_t)tx;
                const size_t slot = (size_t)tm * n->max_off + h_cnt[tm]++;
                h_src[slot] = sm;
                h_j[slot] = j++;
            }
        }
        CUDA_TRY(cudaMemcpyAsync(in_src, h_src.data(), h_src.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(in_j, h_j.data(), h_j.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(in_cnt, h_cnt.data(), h_cnt.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
        v.segidx = segidx;
        v.in_src = in_src;
        v.in_j = in_j;
        v.in_cnt = in_cnt;
    }
    const size_t scratch_bytes = (size_t)n->n_modules * n->max_off * sizeof(double);
    const size_t off_bytes = off.size() * sizeof(int16_t);
    void* scratch = temp(scratch_bytes);
    void* doff = temp(off_bytes);
    if (!scratch || !doff) return fail(SNN_ENOMEM, "device allocation of construction scratch failed");

    CUDA_TRY(cudaMemcpyAsync(doff, off.data(), off_bytes, cudaMemcpyHostToDevice, s));

    b.offsets = (const int16_t*)doff;
    b.scratch = (double*)scratch;
    b.cdf_T = n->cdf_T;
    b.cdf_mod = n->cdf_mod;
    b.cdf_n = n->cdf_n;
    b.segidx = segidx;

    CUDA_TRY(launch_build_cdf(b, s));
    if (pairwise) {
        CUDA_TRY(cudaMemsetAsync(v.td, 0, nsyn * 4, s));  // padding past each row's end
        CUDA_TRY(cudaMemsetAsync(v.w, 0, nsyn * wbytes, s));
        CUDA_TRY(launch_pair_fill(b, v.td, v.w, s));
    } else if (grouped) {
        CUDA_TRY(launch_gen_grouped(b, v.td, v.w, s));
    } else {
        CUDA_TRY(launch_gen_synapses(b, v.td, v.w, s));
    }
    CUDA_TRY(launch_init_state(b, v.V, v.c, v.ref, s));
    if (c.stdp) {
        st = stdp_setup(n, s);
        if (st != SNN_OK) return st;
    }
    CUDA_TRY(cudaMemsetAsync(v.ring, 0, (size_t)n->D * n->Npad * 4, s));
    CUDA_TRY(cudaMemsetAsync(v.seg, 0, (size_t)n->Npad * 4, s));
    CUDA_TRY(cudaMemsetAsync(v.st, 0, sizeof(DevState), s));
    CUDA_TRY(cudaMemsetAsync(v.blk_off, 0, (size_t)(n->nb + 1) * 4, s));
    CUDA_TRY(prepare_deliver(n->nb));
    // the construction buffers must outlive the kernels that read them
    CUDA_TRY(cudaStreamSynchronize(s));
    for (auto& tb : temps) free_block(n, tb.first, tb.second);
    n->grid = deliver_default_grid(n->schedule, n->block, n->nb, v.w_bf16 != 0);
    n->tgrid = grouped ? tiled_grid(v) : 0;
    v.res_quads = persistent_resident_quads(v, n->pgrid);  // neuron state in shared memory during launches
    if (v.segidx) {
        uint32_t chosen = 0;
        st = set_bands(n, 0, &chosen);  // banded delivery when the ring outgrows the L2 budget
        if (st != SNN_OK) return st;
    }
    return SNN_OK;
}

snn_status timed_begin(EventRing& r, cudaStream_t s, int* slot) {
    const int k = (int)(r.next % TIMING_SLOTS);
    if (!r.a[k]) {
        CUDA_TRY(cudaEventCreate(&r.a[k]));
        CUDA_TRY(cudaEventCreate(&r.b[k]));
    }
    if (r.pending[k]) {
        CUDA_TRY(cudaEventSynchronize(r.b[k]));
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, r.a[k], r.b[k]));
        r.total_ms += ms;
        r.count += 1;
        r.pending[k] = false;
    }
    CUDA_TRY(cudaEventRecord(r.a[k], s));
    *slot = k;
    return SNN_OK;
}

snn_status timed_end(EventRing& r, cudaStream_t s, int k) {
    CUDA_TRY(cudaEventRecord(r.b[k], s));
    r.pending[k] = true;
    r.next += 1;
    return SNN_OK;
}

snn_status drain(EventRing& r) {
    for (int k = 0; k < TIMING_SLOTS; ++k) {
        if (!r.pending[k]) continue;
        CUDA_TRY(cudaEventSynchronize(r.b[k]));
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, r.a[k], r.b[k]));
        r.total_ms += ms;
        r.count += 1;
        r.pending[k] = false;
    }
    return SNN_OK;
}

struct SnapshotHeader {
    uint64_t magic;
    uint32_t version, N, Npad, D;
    uint64_t seed;
    uint32_t K, pad;
};
constexpr uint64_t SNAP_MAGIC = 0x31504E5350534E53ull;  // "SNSPSNP1"

}  // namespace

const snn_config* snn_config_of(const snn_net* net) { return &net->cfg; }

cudaError_t snn_set_raster_count(snn_net* net, uint64_t count, cudaStream_t s) {
    static thread_local uint64_t staged;  // pageable source: copied before the call returns
    staged = count;
    cudaError_t e = cudaMemcpyAsync(&net->v.st->raster_count, &staged, sizeof staged, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

extern "C" {

const char* snn_last_error(void) { return g_last_error.c_str(); }

uint64_t snn_launch_count(void) { return g_launches.load(); }

snn_status snn_build_network(const snn_config* cfg, snn_alloc_fn alloc_fn, snn_free_fn free_fn,
                             void* alloc_ctx, void* stream, snn_net** out) {
    if (!out) return fail(SNN_EINVAL, "out is NULL");
    *out = nullptr;
    snn_status st = validate(cfg);
    if (st != SNN_OK) return st;
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return fail(SNN_EINVAL, "alloc_fn and free_fn must both be set or both be NULL");
    snn_net* n = new (std::nothrow) snn_net();
    if (!n) return fail(SNN_ENOMEM, "host allocation failed");
    n->cfg = *cfg;
    n->alloc_fn = alloc_fn;
    n->free_fn = free_fn;
    n->alloc_ctx = alloc_ctx;
    cudaGetDevice(&n->device);
    NvtxRange range("snn_build_network");
    st = build_impl(n, (cudaStream_t)stream);
    if (st != SNN_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        release_all(n);
        delete n;
        return st;
    }
    *out = n;
    return SNN_OK;
}

snn_status snn_step(snn_net* n, uint32_t n_steps, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    NvtxRange range("snn_step");
    cudaStream_t s = (cudaStream_t)stream;
    if (n->schedule >= 2) {
        // one cooperative launch per call (in pieces of at most 2^20 steps)
        for (uint32_t done = 0; done < n_steps;) {
            const uint32_t m = std::min<uint32_t>(n_steps - done, 1u << 20);
            CUDA_TRY(cudaMemsetAsync(&n->v.st->bar_count, 0, sizeof(uint32_t), s));
            if (n->schedule == 3)
                CUDA_TRY(cudaMemsetAsync(n->v.mod_cnt, 0, (size_t)n->n_modules * 2 * 4, s));
            int slot = 0;
            const bool timed = n->timing_every > 0;
            if (timed) {
                snn_status st = timed_begin(n->ev_persist, s, &slot);
                if (st != SNN_OK) return st;
            }
            NvtxRange lr(n->schedule == 3   ? "persistent: target tiles"
                         : n->schedule == 4 ? "persistent: owned windows"
                         : n->schedule == 5 ? "persistent: pulled windows"
                                            : "persistent: neuron + delivery phases");
            if (n->schedule == 3)
                CUDA_TRY(launch_tiled(n->v, m, n->tgrid, s));
            else if (n->schedule == 4)
                CUDA_TRY(launch_owned(n->v, m, n->ogrid, s));
            else if (n->schedule == 5)
                CUDA_TRY(launch_pull(n->v, m, n->plgrid, s));
            else
                CUDA_TRY(launch_persistent(n->v, m, n->pgrid, s));
            if (timed) {
                snn_status st = timed_end(n->ev_persist, s, slot);
                if (st != SNN_OK) return st;
            }
            done += m;
        }
        return SNN_OK;
    }
    for (uint32_t k = 0; k < n_steps; ++k) {
        int slot = 0;
        const bool timed = n->timing_every > 0 && (n->step_calls++ % (uint64_t)n->timing_every) == 0;
        if (timed) {
            snn_status st = timed_begin(n->ev_neuron, s, &slot);
            if (st != SNN_OK) return st;
        }
        {
            NvtxRange r("neuron phase");
            CUDA_TRY(launch_neuron_step(n->v, s));
            if (n->stdp) CUDA_TRY(launch_stdp_pre_delivery(n->v, n->sp, s));
        }
        if (timed) {
            snn_status st = timed_end(n->ev_neuron, s, slot);
            if (st == SNN_OK) st = timed_begin(n->ev_deliver, s, &slot);
            if (st != SNN_OK) return st;
        }
        {
            NvtxRange r("delivery phase");
            CUDA_TRY(launch_deliver(n->v, n->schedule, n->block, n->grid, s));
            if (n->stdp) CUDA_TRY(launch_stdp_apply(n->v, n->sp, s));
        }
        if (timed) {
            snn_status st = timed_end(n->ev_deliver, s, slot);
            if (st != SNN_OK) return st;
        }
    }
    return SNN_OK;
}

snn_status snn_read_spikes(snn_net* n, uint32_t* steps, uint32_t* ids, size_t cap, size_t* n_out,
                           void* stream) {
    if (!n || !n_out) return fail(SNN_EINVAL, "net or n_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    DevState ds;
    CUDA_TRY(cudaMemcpyAsync(&ds, n->v.st, sizeof ds, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    uint64_t avail = ds.raster_count < n->v.raster_cap ? ds.raster_count : n->v.raster_cap;
    const size_t m = (size_t)(avail < cap ? avail : cap);
    if (m && steps) CUDA_TRY(cudaMemcpyAsync(steps, n->v.raster_t, m * 4, cudaMemcpyDeviceToHost, s));
    if (m && ids) CUDA_TRY(cudaMemcpyAsync(ids, n->v.raster_id, m * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *n_out = m;
    if (ds.err & ERR_BOUNDS) return fail(SNN_ECUDA, "a device bounds check failed (error bits 0x%x)", ds.err);
    if (ds.err) return fail(SNN_ETIMEOUT, "a device-side wait ran out or a device check failed (error bits 0x%x)", ds.err);
    if (ds.raster_count > n->v.raster_cap)
        return fail(SNN_EOVERFLOW, "raster overflow: %llu spikes recorded, capacity %llu",
                    (unsigned long long)ds.raster_count, (unsigned long long)n->v.raster_cap);
    return SNN_OK;
}

snn_status snn_clear_raster(snn_net* n, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    CUDA_TRY(cudaMemsetAsync(&n->v.st->raster_count, 0, sizeof(uint64_t), (cudaStream_t)stream));
    return SNN_OK;
}

snn_status snn_get_stats(snn_net* n, snn_stats* out, void* stream) {
    if (!n || !out) return fail(SNN_EINVAL, "net or out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    DevState ds;
    CUDA_TRY(cudaMemcpyAsync(&ds, n->v.st, sizeof ds, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    out->steps = ds.t;
    out->n_spikes = ds.n_spikes;
    out->rec_events = ds.rec_events;
    out->ext_events = ds.ext_events;
    out->raster_count = ds.raster_count;
    out->raster_capacity = n->v.raster_cap;
    out->neuron_phase_ns = ds.phase_ns[0];
    out->deliver_phase_ns = ds.phase_ns[1];
    if (ds.err & ERR_BOUNDS) return fail(SNN_ECUDA, "a device bounds check failed (error bits 0x%x)", ds.err);
    if (ds.err) return fail(SNN_ETIMEOUT, "a device-side wait ran out or a device check failed (error bits 0x%x)", ds.err);
    return SNN_OK;
}

snn_status snn_get_dims(snn_net* n, uint32_t* N, uint32_t* K, uint32_t* D, uint64_t* bytes) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if (N) *N = n->N;
    if (K) *K = n->K;
    if (D) *D = n->D;
    if (bytes) *bytes = n->device_bytes;
    return SNN_OK;
}

snn_status snn_get_rows(snn_net* n, uint32_t first, uint32_t count, uint32_t* tgt, float* w, uint8_t* d,
                        void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if ((uint64_t)first + count > n->N) return fail(SNN_EINVAL, "rows [%u, %u) out of range", first, first + count);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rows = count, Kp = n->Kpad;
    const size_t e0 = (size_t)first * Kp;
    // copy the padded rows, keep each row's first len entries; split target | delay << 24
    std::vector<uint32_t> len(rows, n->K);
    if (n->v.row_len && rows)
        CUDA_TRY(cudaMemcpyAsync(len.data(), n->v.row_len + first, rows * 4, cudaMemcpyDeviceToHost, s));
    const bool bf = n->v.w_bf16 != 0;
    std::vector<uint32_t> td((tgt || d) ? rows * Kp : 0);
    std::vector<uint32_t> wr(w && !bf ? rows * Kp : 0);  // f32 bits
    std::vector<uint16_t> wh(w && bf ? rows * Kp : 0);   // bf16 bits
    if ((tgt || d) && rows && Kp)
        CUDA_TRY(cudaMemcpyAsync(td.data(), n->v.td + e0, rows * Kp * 4, cudaMemcpyDeviceToHost, s));
    if (w && rows && Kp) {
        if (bf)
            CUDA_TRY(cudaMemcpyAsync(wh.data(), (const uint16_t*)n->v.w + e0, rows * Kp * 2, cudaMemcpyDeviceToHost, s));
        else
            CUDA_TRY(cudaMemcpyAsync(wr.data(), (const float*)n->v.w + e0, rows * Kp * 4, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    size_t o = 0;
    for (size_t r = 0; r < rows; ++r) {
        for (size_t k = 0; k < len[r]; ++k, ++o) {
            const size_t e = r * Kp + k;
            if (tgt) tgt[o] = td[e] & 0xFFFFFFu;
            if (d) d[o] = (uint8_t)(td[e] >> 24);
            if (w) {
                const uint32_t bits = bf ? (uint32_t)wh[e] << 16 : wr[e];
                std::memcpy(&w[o], &bits, 4);
            }
        }
    }
    return SNN_OK;
}

snn_status snn_get_row_lengths(snn_net* n, uint32_t first, uint32_t count, uint32_t* len, void* stream) {
    if (!n || !len) return fail(SNN_EINVAL, "net or len is NULL");
    if ((uint64_t)first + count > n->N) return fail(SNN_EINVAL, "rows [%u, %u) out of range", first, first + count);
    if (!n->v.row_len) {
        for (uint32_t r = 0; r < count; ++r) len[r] = n->K;
        return SNN_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (count) CUDA_TRY(cudaMemcpyAsync(len, n->v.row_len + first, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_get_stdp(snn_net* n, int32_t* delta, float* y, float* x, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if (!n->stdp) return fail(SNN_EINVAL, "the network has no plasticity (stdp = 0)");
    cudaStream_t s = (cudaStream_t)stream;
    if (delta) {
        std::vector<uint32_t> len(n->N);
        snn_status st = snn_get_row_lengths(n, 0, n->N, len.data(), stream);
        if (st != SNN_OK) return st;
        std::vector<int32_t> all((size_t)n->N * n->Kpad);
        CUDA_TRY(cudaMemcpyAsync(all.data(), n->sp.delta, all.size() * 4, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        size_t o = 0;
        for (uint32_t i = 0; i < n->N; ++i) {
            std::memcpy(delta + o, all.data() + (size_t)i * n->Kpad, (size_t)len[i] * 4);
            o += len[i];
        }
    }
    if (y) CUDA_TRY(cudaMemcpyAsync(y, n->sp.y, (size_t)n->N * 4, cudaMemcpyDeviceToHost, s));
    if (x) CUDA_TRY(cudaMemcpyAsync(x, n->sp.x, (size_t)n->N * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_construction_tables(const snn_config* cfg, float* wtab, uint64_t* dthr, uint32_t* n_dthr,
                                   int32_t* pair_dx, int32_t* pair_dy, uint64_t* pair_thr, uint32_t cap,
                                   uint32_t* n_pair) {
    snn_status st = validate(cfg);
    if (st != SNN_OK) return st;
    HostTables t;
    host_tables(*cfg, &t);
    if (wtab && !t.wtab.empty()) std::memcpy(wtab, t.wtab.data(), t.wtab.size() * 4);
    if (n_dthr) *n_dthr = (uint32_t)t.dthr.size();
    if (dthr && !t.dthr.empty()) std::memcpy(dthr, t.dthr.data(), t.dthr.size() * 8);
    if (n_pair) *n_pair = (uint32_t)t.pdx.size();
    if (pair_dx || pair_dy || pair_thr) {
        if (t.pdx.size() > cap) return fail(SNN_EINVAL, "stencil of %zu entries exceeds cap %u", t.pdx.size(), cap);
        for (size_t k = 0; k < t.pdx.size(); ++k) {
            if (pair_dx) pair_dx[k] = t.pdx[k];
            if (pair_dy) pair_dy[k] = t.pdy[k];
            if (pair_thr) pair_thr[k] = t.pthr[k];
        }
    }
    return SNN_OK;
}

snn_status snn_get_segments(snn_net* n, uint32_t first, uint32_t count, uint16_t* seg, uint32_t* stride,
                            void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if (stride) *stride = n->v.seg_stride;
    if (!seg) return SNN_OK;
    if (!n->v.segidx) return fail(SNN_EINVAL, "the network has no segment index (grouped layout or pairwise law)");
    if ((uint64_t)first + count > n->N) return fail(SNN_EINVAL, "rows out of range");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(seg, n->v.segidx + (size_t)first * n->v.seg_stride,
                             (size_t)count * n->v.seg_stride * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_get_table(snn_net* n, uint32_t* tgt, float* w, uint8_t* d, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    return snn_get_rows(n, 0, n->N, tgt, w, d, stream);
}

snn_status snn_get_cdf(snn_net* n, uint32_t* thresh, uint32_t* tgt_module, uint32_t* counts,
                       uint32_t* max_offsets, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t tot = (size_t)n->n_modules * n->max_off;
    if (max_offsets) *max_offsets = n->max_off;
    if (thresh) CUDA_TRY(cudaMemcpyAsync(thresh, n->cdf_T, tot * 4, cudaMemcpyDeviceToHost, s));
    if (tgt_module) CUDA_TRY(cudaMemcpyAsync(tgt_module, n->cdf_mod, tot * 4, cudaMemcpyDeviceToHost, s));
    if (counts) CUDA_TRY(cudaMemcpyAsync(counts, n->cdf_n, (size_t)n->n_modules * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_get_state(snn_net* n, float* V, float* c, uint8_t* ref, int32_t* ring, uint32_t* t,
                         void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = n->N;
    if (V) CUDA_TRY(cudaMemcpyAsync(V, n->v.V, N * 4, cudaMemcpyDeviceToHost, s));
    if (c) CUDA_TRY(cudaMemcpyAsync(c, n->v.c, N * 4, cudaMemcpyDeviceToHost, s));
    if (ref) CUDA_TRY(cudaMemcpyAsync(ref, n->v.ref, N, cudaMemcpyDeviceToHost, s));
    if (ring && N)
        CUDA_TRY(cudaMemcpy2DAsync(ring, N * 4, n->v.ring, (size_t)n->Npad * 4, N * 4, n->D,
                                   cudaMemcpyDeviceToHost, s));
    DevState ds;
    CUDA_TRY(cudaMemcpyAsync(&ds, n->v.st, sizeof ds, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (t) *t = ds.t;
    return SNN_OK;
}

snn_status snn_set_state(snn_net* n, const float* V, const float* c, const uint8_t* ref, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = n->N;
    if (V) CUDA_TRY(cudaMemcpyAsync(n->v.V, V, N * 4, cudaMemcpyHostToDevice, s));
    if (c) CUDA_TRY(cudaMemcpyAsync(n->v.c, c, N * 4, cudaMemcpyHostToDevice, s));
    if (ref) CUDA_TRY(cudaMemcpyAsync(n->v.ref, ref, N, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_snapshot(snn_net* n, void* host_buf, size_t cap, size_t* nbytes, void* stream) {
    if (n && n->stdp) return fail(SNN_EINVAL, "snapshots do not hold the plastic weights of a network with stdp");
    if (!n || !nbytes) return fail(SNN_EINVAL, "net or n is NULL");
    const size_t N = n->Npad, D = n->D;
    const size_t need = sizeof(SnapshotHeader) + sizeof(DevState) + N * 4 * 2 + N + D * N * 4;
    *nbytes = need;
    if (!host_buf) return SNN_OK;
    if (cap < need) return fail(SNN_EINVAL, "snapshot buffer too small (%zu < %zu)", cap, need);
    cudaStream_t s = (cudaStream_t)stream;
    char* p = (char*)host_buf;
    SnapshotHeader h{SNAP_MAGIC, 1u, n->N, n->Npad, n->D, n->cfg.seed, n->K, 0u};
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    CUDA_TRY(cudaMemcpyAsync(p, n->v.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    p += sizeof(DevState);
    CUDA_TRY(cudaMemcpyAsync(p, n->v.V, N * 4, cudaMemcpyDeviceToHost, s));
    p += N * 4;
    CUDA_TRY(cudaMemcpyAsync(p, n->v.c, N * 4, cudaMemcpyDeviceToHost, s));
    p += N * 4;
    CUDA_TRY(cudaMemcpyAsync(p, n->v.ref, N, cudaMemcpyDeviceToHost, s));
    p += N;
    CUDA_TRY(cudaMemcpyAsync(p, n->v.ring, D * N * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_restore(snn_net* n, const void* host_buf, size_t nbytes, void* stream) {
    if (n && n->stdp) return fail(SNN_EINVAL, "snapshots do not hold the plastic weights of a network with stdp");
    if (!n || !host_buf) return fail(SNN_EINVAL, "net or buffer is NULL");
    const size_t N = n->Npad, D = n->D;
    const size_t need = sizeof(SnapshotHeader) + sizeof(DevState) + N * 4 * 2 + N + D * N * 4;
    if (nbytes != need) return fail(SNN_EINVAL, "snapshot size mismatch (%zu != %zu)", nbytes, need);
    const char* p = (const char*)host_buf;
    SnapshotHeader h;
    std::memcpy(&h, p, sizeof h);
    if (h.magic != SNAP_MAGIC || h.version != 1u || h.N != n->N || h.Npad != n->Npad || h.D != n->D ||
        h.seed != n->cfg.seed || h.K != n->K)
        return fail(SNN_EINVAL, "snapshot was taken from a different network");
    p += sizeof h;
    DevState ds;
    std::memcpy(&ds, p, sizeof ds);
    ds.done = 0;
    ds.raster_count = 0;  // recorded spikes are not part of the state
    ds.raster_base = 0;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(n->v.st, &ds, sizeof ds, cudaMemcpyHostToDevice, s));
    p += sizeof(DevState);
    CUDA_TRY(cudaMemcpyAsync(n->v.V, p, N * 4, cudaMemcpyHostToDevice, s));
    p += N * 4;
    CUDA_TRY(cudaMemcpyAsync(n->v.c, p, N * 4, cudaMemcpyHostToDevice, s));
    p += N * 4;
    CUDA_TRY(cudaMemcpyAsync(n->v.ref, p, N, cudaMemcpyHostToDevice, s));
    p += N;
    CUDA_TRY(cudaMemcpyAsync(n->v.ring, p, D * N * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_set_window(snn_net* n, uint32_t window, uint32_t queue_cap, uint32_t* window_out,
                          uint32_t* cap_out, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));  // no launch in flight uses the queues
    snn_status st = owned_setup(n, window, queue_cap);
    if (st != SNN_OK) return st;
    if (window_out) *window_out = n->v.own_W;
    if (cap_out) *cap_out = n->v.own_cap;
    return SNN_OK;
}

snn_status snn_set_pull_window(snn_net* n, uint32_t window, int32_t band_mode, uint32_t* window_out,
                               int32_t* mode_out, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));  // no launch in flight uses the run table
    snn_status st = pull_setup(n, window, band_mode);
    if (st != SNN_OK) return st;
    if (window_out) *window_out = n->v.pull_W;
    if (mode_out) *mode_out = n->pull_mode;
    return SNN_OK;
}

snn_status snn_set_bands(snn_net* n, uint32_t bands, uint32_t* chosen, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));  // no launch in flight reads the tables
    return set_bands(n, bands, chosen);
}

snn_status snn_set_resident_state(snn_net* n, int32_t enable, int32_t* resident, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if (enable != 0 && enable != 1) return fail(SNN_EINVAL, "enable must be 0 or 1");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));  // no launch in flight uses the old view
    n->v.res_quads = enable ? persistent_resident_quads(n->v, n->pgrid) : 0u;
    if (resident) *resident = n->v.res_quads > 0 ? 1 : 0;
    return SNN_OK;
}

snn_status snn_set_schedule(snn_net* n, int32_t schedule, int32_t block) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if (schedule < 0 || schedule > 5) return fail(SNN_EINVAL, "schedule must be 0, 1, 2, 3, 4 or 5");
    if (n->stdp && schedule >= 2)
        return fail(SNN_EINVAL, "a network with stdp runs the per-step schedules 0 and 1 only");
    if (schedule == 4 && n->ogrid == 0) {
        snn_status st = owned_setup(n, 0, 0);
        if (st != SNN_OK) return st;
    }
    if (schedule == 5 && n->plgrid == 0) {
        snn_status st = pull_setup(n, 0, 0);
        if (st != SNN_OK) return st;
    }
    if (schedule == 3 && n->cfg.table_layout != SNN_LAYOUT_GROUPED)
        return fail(SNN_EINVAL, "schedule 3 needs a network built with table_layout = SNN_LAYOUT_GROUPED");
    if (schedule == 3 && n->tgrid == 0)
        return fail(SNN_EINVAL, "schedule 3: the (D - 1) x M delivery tile does not fit in shared memory");
    if (block == 0) block = 256;
    if (block < 32 || block > 256 || block % 32) return fail(SNN_EINVAL, "block must be a multiple of 32 in [32, 256]");
    n->schedule = schedule;
    if (schedule < 2) {
        n->block = block;
        n->grid = deliver_default_grid(schedule, block, n->nb, n->v.w_bf16 != 0);
    }
    return SNN_OK;
}

snn_status snn_set_timing(snn_net* n, int32_t every) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if (every < 0) return fail(SNN_EINVAL, "every must be >= 0");
    n->timing_every = every;
    n->step_calls = 0;
    return SNN_OK;
}

snn_status snn_kernel_time(snn_net* n, int32_t which, double* ms, uint64_t* launches) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    EventRing* r = which == SNN_TIMER_NEURON ? &n->ev_neuron
                 : which == SNN_TIMER_DELIVER ? &n->ev_deliver
                 : which == SNN_TIMER_PERSISTENT ? &n->ev_persist : nullptr;
    if (!r) return fail(SNN_EINVAL, "unknown timer %d", which);
    snn_status st = drain(*r);
    if (st != SNN_OK) return st;
    if (ms) *ms = r->total_ms;
    if (launches) *launches = r->count;
    return SNN_OK;
}

snn_status snn_set_wait_limit(snn_net* n, uint64_t ns) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    if (ns == 0) return fail(SNN_EINVAL, "the wait limit must be positive");
    n->v.wait_limit_ns = ns;
    return SNN_OK;
}

snn_status snn_set_barrier_extra(snn_net* n, uint32_t extra) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    n->v.barrier_extra = extra;
    return SNN_OK;
}

snn_status snn_clear_error(snn_net* n, void* stream) {
    if (!n) return fail(SNN_EINVAL, "net is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(&n->v.st->err, 0, sizeof(uint32_t), s));
    CUDA_TRY(cudaMemsetAsync(&n->v.st->bar_count, 0, sizeof(uint32_t), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

void snn_destroy(snn_net* n) {
    if (!n) return;
    cudaDeviceSynchronize();
    destroy_events(n->ev_deliver);
    destroy_events(n->ev_neuron);
    destroy_events(n->ev_persist);
    release_all(n);
    delete n;
}

// ---------------------------------------------------------------------------
// Batched execution.

// A wave: networks advanced together by one cooperative launch, either in
// one global neuron / task space (meta) or each on a group of CTAs (gmeta).
struct BatchWave {
    BatchMeta meta{};
    GroupMeta gmeta{};
    uint32_t first = 0, count = 0;
    int grid = 0;
    int shape = 0;  // global waves: launch shape of k_run_batch
    bool grouped = false;
    uint32_t stage_off = 0;  // grouped: offset of the wave's CTA prefix in the staging words
};

struct snn_batch {
    std::vector<snn_net*> nets;
    snn_alloc_fn alloc_fn = nullptr;
    snn_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;
    std::vector<void*> blocks;
    std::vector<BatchWave> waves;
    // staging words: the steps of every network (n), then the CTA prefix of
    // every grouped wave (count + 1 each, at most 2 n in all)
    uint32_t* d_steps = nullptr;
    uint32_t* h_steps = nullptr;  // pinned
    uint32_t stage_len = 0;
    uint64_t* d_gns = nullptr;  // per network: ns its group took in the last call
    uint64_t* h_gns = nullptr;  // pinned copy, read back by the next call
    std::vector<double> work;   // per network: estimated CTA-microseconds of one step
    std::vector<uint32_t> last_cta, last_steps;  // CTAs and steps of each network's group in the last call
    int32_t mode = SNN_BATCH_GROUPS;
    int32_t shape = 0;  // launch shape of global waves (batch_kernels.cu)
    int ggrid = 0;  // grouped kernel's grid
    uint64_t ring_budget = 0;
    bool use_graph = false;
    bool graph_valid = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<uint32_t> graph_key;  // longest step count of each wave when the graph was captured
    EventRing ev;
};

namespace {

void* batch_alloc(snn_batch* b, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (b->alloc_fn) {
        p = b->alloc_fn(bytes, b->alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) b->blocks.push_back(p);
    return p;
}

uint64_t ring_bytes(const snn_net* n) { return (uint64_t)n->D * n->Npad * 4; }

// Cost model of a grouped network: one step on G CTAs takes about
// GROUP_FIXED_US + W / G microseconds, W the step's work in CTA-microseconds.
// The fixed part is the latency chain of a step (two grid barriers, the
// offset scan, dependent loads), which a group pays whatever its size.
constexpr double GROUP_FIXED_US = 8.0;
constexpr double NEURON_US = 8e-6;  // neuron update on the whole GPU, per neuron
constexpr double EVENT_US = 1.0 / 1.9e5;  // delivery on the whole GPU, per synaptic event

// Work before any measurement: the imposed spike rate (10 Hz if none) times
// the out-degree (the longest row under the per-pair law).
double initial_work(const snn_net* n, int grid) {
    const double rate = n->cfg.imposed_rate_hz > 0 ? n->cfg.imposed_rate_hz : 10.0;
    const double events = (double)n->N * rate * n->cfg.dt_ms * 1e-3 * n->K;
    return std::max(grid, 1) * (NEURON_US * n->N + EVENT_US * events);
}

// CTAs of a grouped wave: network i (s[i] steps, work W[i]) on G_i CTAs takes
// about s_i (F + W_i / G_i).  The smallest makespan T whose groups fit in S
// CTAs is found by bisection (G_i = ceil(s_i W_i / (T - s_i F)), at least 1),
// then the CTAs left over go one at a time to the group that would finish
// last.  Idle networks (s_i = 0) get none.  Writes the prefix gcta[0..count].
void partition_groups(const uint32_t* s, const double* W, uint32_t count, uint32_t S, uint32_t* G, uint32_t* gcta) {
    const double F = GROUP_FIXED_US;
    auto need = [&](double T, bool write) {
        uint64_t total = 0;
        for (uint32_t i = 0; i < count; ++i) {
            uint32_t g = 0;
            if (s[i] > 0) {
                const double x = s[i] * W[i] / (T - s[i] * F);
                g = x >= S ? S : std::max(1u, (uint32_t)std::ceil(x));
            }
            if (write) G[i] = g;
            total += g;
        }
        return total;
    };
    double lo = 0, hi = 0;
    for (uint32_t i = 0; i < count; ++i) {
        if (s[i] == 0) continue;
        lo = std::max(lo, s[i] * (F + W[i] / S));
        hi = std::max(hi, s[i] * (F + W[i]));
    }
    if (hi > 0) {
        for (int it = 0; it < 60 && hi - lo > 1e-9 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (need(mid, false) <= S)
                hi = mid;
            else
                lo = mid;
        }
    }
    uint64_t used = need(hi * (1 + 1e-12), true);
    while (used < S) {
        uint32_t best = count;
        double tb = -1;
        for (uint32_t i = 0; i < count; ++i) {
            if (G[i] == 0) continue;
            const double t = s[i] * (F + W[i] / G[i]);
            if (t > tb) {
                tb = t;
                best = i;
            }
        }
        if (best == count) break;
        ++G[best];
        ++used;
    }
    gcta[0] = 0;
    for (uint32_t i = 0; i < count; ++i) gcta[i + 1] = gcta[i] + G[i];
}

// Device tables of one wave: networks [first, first + count).
snn_status build_wave(snn_batch* b, uint32_t first, uint32_t count, BatchWave* w) {
    snn_net* const* nets = b->nets.data() + first;
    bool group = b->mode != SNN_BATCH_GLOBAL && count >= 2 && b->ggrid > 0 && count <= (uint32_t)b->ggrid;
    for (uint32_t i = 0; i < count && group; ++i) group = nets[i]->v.n_bands <= 1;
    if (group) {
        NetView* d_views = (NetView*)batch_alloc(b, count * sizeof(NetView));
        if (!d_views) return fail(SNN_ENOMEM, "batch allocation failed");
        std::vector<NetView> views(count);
        for (uint32_t i = 0; i < count; ++i) {
            views[i] = nets[i]->v;
            views[i].res_quads = 0;  // sized for the network's own grid, not for a group
        }
        CUDA_TRY(cudaMemcpy(d_views, views.data(), count * sizeof(NetView), cudaMemcpyHostToDevice));
        w->grouped = true;
        w->first = first;
        w->count = count;
        w->grid = b->ggrid;
        w->gmeta.views = d_views;
        w->gmeta.steps = b->d_steps + first;
        w->gmeta.gns = b->d_gns + first;
        w->gmeta.n = count;
        return SNN_OK;  // the CTA prefix is placed by the caller
    }
    uint64_t Qtot = 0, tasks = 0;
    for (uint32_t i = 0; i < count; ++i) {
        Qtot += nets[i]->Npad / 4;
        tasks += (uint64_t)nets[i]->N * ((nets[i]->K + 127) / 128);
    }
    if (Qtot >= (1ull << 32) || tasks >= (1ull << 32)) return fail(SNN_EINVAL, "a batch wave is too large");
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = batch_grid(count, (uint32_t)(8 * PERSIST_WARPS * sms) + count, b->shape);
    if (grid <= 0) return fail(SNN_EINVAL, "the batch kernel does not fit on this device (%u networks)", count);
    // global quad offsets; first and last warp overlapping each network
    const uint64_t TW = (uint64_t)grid * PERSIST_WARPS;
    std::vector<uint32_t> qoff(count + 1, 0), wlo(count, 0), cbase(count + 1, 0);
    for (uint32_t i = 0; i < count; ++i) qoff[i + 1] = qoff[i] + nets[i]->Npad / 4;
    auto owner = [&](uint64_t q) {  // the warp whose range [Qtot w / TW, Qtot (w+1) / TW) holds quad q
        uint64_t lo = 0, hi = TW;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) / 2;
            if (Qtot * mid / TW <= q)
                lo = mid;
            else
                hi = mid;
        }
        return (uint32_t)lo;
    };
    for (uint32_t i = 0; i < count; ++i) {
        wlo[i] = owner(qoff[i]);
        const uint32_t whi = owner(qoff[i + 1] - 1);
        cbase[i + 1] = cbase[i] + (whi - wlo[i] + 1);
    }
    const uint32_t n_seg = cbase[count];
    NetView* d_views = (NetView*)batch_alloc(b, count * sizeof(NetView));
    uint32_t* d_qoff = (uint32_t*)batch_alloc(b, (count + 1) * 4);
    uint32_t* d_cbase = (uint32_t*)batch_alloc(b, (count + 1) * 4);
    uint32_t* d_wlo = (uint32_t*)batch_alloc(b, count * 4);
    uint32_t* d_wcnt = (uint32_t*)batch_alloc(b, (size_t)n_seg * 4);
    DevState* d_st = (DevState*)batch_alloc(b, sizeof(DevState));
    if (!d_views || !d_qoff || !d_cbase || !d_wlo || !d_wcnt || !d_st) return fail(SNN_ENOMEM, "batch allocation failed");
    std::vector<NetView> views(count);
    uint64_t limit = ~0ull;
    uint32_t extra = 0;
    for (uint32_t i = 0; i < count; ++i) {
        views[i] = nets[i]->v;
        limit = std::min(limit, nets[i]->v.wait_limit_ns);
        extra = std::max(extra, nets[i]->v.barrier_extra);
    }
    cudaError_t e = cudaMemcpy(d_views, views.data(), count * sizeof(NetView), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_qoff, qoff.data(), (count + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_cbase, cbase.data(), (count + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_wlo, wlo.data(), count * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_wcnt, 0, (size_t)n_seg * 4);
    if (e == cudaSuccess) e = cudaMemset(d_st, 0, sizeof(DevState));
    if (e != cudaSuccess) return fail(SNN_ECUDA, "batch set-up: %s", cudaGetErrorString(e));
    BatchMeta& m = w->meta;
    m.views = d_views;
    m.qoff = d_qoff;
    m.cbase = d_cbase;
    m.wlo = d_wlo;
    m.wcnt = d_wcnt;
    m.steps = b->d_steps + first;
    m.bst = d_st;
    m.wait_limit_ns = limit;
    m.barrier_extra = extra;
    m.n = count;
    m.n_seg = n_seg;
    m.Qtot = (uint32_t)Qtot;
    w->first = first;
    w->count = count;
    w->grid = grid;
    w->shape = b->shape;
    return SNN_OK;
}

}  // namespace

snn_status snn_batch_create(snn_net* const* nets, uint32_t n, snn_alloc_fn alloc_fn, snn_free_fn free_fn,
                            void* alloc_ctx, snn_batch** out) {
    if (!out || !nets || n == 0) return fail(SNN_EINVAL, "nets, n and out must be set");
    *out = nullptr;
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return fail(SNN_EINVAL, "alloc_fn and free_fn must both be set or both be NULL");
    for (uint32_t i = 0; i < n; ++i) {
        if (!nets[i]) return fail(SNN_EINVAL, "network %u is NULL", i);
        for (uint32_t j = 0; j < i; ++j)
            if (nets[j] == nets[i]) return fail(SNN_EINVAL, "network %u appears twice", i);
        if (nets[i]->stdp) return fail(SNN_EINVAL, "network %u has stdp, which batches do not run", i);
    }
    snn_batch* b = new (std::nothrow) snn_batch();
    if (!b) return fail(SNN_ENOMEM, "host allocation failed");
    b->nets.assign(nets, nets + n);
    b->alloc_fn = alloc_fn;
    b->free_fn = free_fn;
    b->alloc_ctx = alloc_ctx;
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    b->ring_budget = l2 > 0 ? (uint64_t)l2 / 2 : (64ull << 20);
    b->d_steps = (uint32_t*)batch_alloc(b, (size_t)n * 12);
    b->d_gns = (uint64_t*)batch_alloc(b, (size_t)n * 8);
    if (!b->d_steps || !b->d_gns || cudaMallocHost(&b->h_steps, (size_t)n * 12) != cudaSuccess ||
        cudaMallocHost(&b->h_gns, (size_t)n * 8) != cudaSuccess) {
        cudaGetLastError();
        snn_batch_destroy(b);
        return fail(SNN_ENOMEM, "batch allocation failed");
    }
    std::memset(b->h_gns, 0, (size_t)n * 8);  // no measured group time yet
    b->ggrid = groups_grid();
    b->work.resize(n);
    b->last_cta.assign(n, 0);
    b->last_steps.assign(n, 0);
    for (uint32_t i = 0; i < n; ++i) b->work[i] = initial_work(b->nets[i], b->ggrid);
    snn_status st = snn_batch_set_ring_budget(b, b->ring_budget);
    if (st != SNN_OK) {
        snn_batch_destroy(b);
        return st;
    }
    *out = b;
    return SNN_OK;
}

snn_status snn_batch_set_ring_budget(snn_batch* b, uint64_t bytes) {
    if (!b || bytes == 0) return fail(SNN_EINVAL, "batch is NULL or the budget is 0");
    CUDA_TRY(cudaDeviceSynchronize());  // tables of the old waves may still be in use
    b->ring_budget = bytes;
    b->waves.clear();
    b->graph_valid = false;
    const uint32_t n = (uint32_t)b->nets.size();
    uint32_t stage = n;  // staging words taken: the steps, then the CTA prefixes
    // waves of consecutive networks whose delay rings fit together in the budget
    for (uint32_t first = 0; first < n;) {
        uint64_t used = ring_bytes(b->nets[first]);
        uint32_t count = 1;
        while (first + count < n && used + ring_bytes(b->nets[first + count]) <= b->ring_budget)
            used += ring_bytes(b->nets[first + count++]);
        BatchWave w;
        snn_status st = build_wave(b, first, count, &w);
        if (st != SNN_OK) return st;
        if (w.grouped) {
            w.stage_off = stage;
            w.gmeta.gcta = b->d_steps + stage;
            stage += count + 1;
        }
        b->waves.push_back(w);
        first += count;
    }
    b->stage_len = stage;
    return SNN_OK;
}

// Autotuner of a batch: every (layout, launch shape, ring budget) candidate is
// timed on `trial_steps` steps of every network from one snapshot of all of
// their states (a first call refines the grouped layout's cost model, the
// second is timed), the states are restored after each, and the fastest is
// kept.  Candidates that give the same wave plan as an earlier one are not
// run again.  The choice is cached in a text file keyed by the GPU and the
// networks' shapes.
snn_status snn_batch_autotune(snn_batch* b, uint32_t trial_steps, const char* cache_path, int32_t* mode_out,
                              int32_t* shape_out, uint64_t* budget_out, double* best_ms, double* trial_ms,
                              void* stream) {
    if (trial_ms)
        for (int k = 0; k < SNN_BATCH_TUNE_CANDIDATES; ++k) trial_ms[k] = -1.0;
    if (!b || trial_steps == 0) return fail(SNN_EINVAL, "batch is NULL or trial_steps is 0");
    NvtxRange range("snn_batch_autotune");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)b->nets.size();
    for (snn_net* net : b->nets)
        if (net->stdp) return fail(SNN_EINVAL, "a network of the batch has stdp");
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the networks' shapes
    auto mix = [&](uint64_t x) {
        for (int k = 0; k < 8; ++k) {
            h ^= (x >> (8 * k)) & 0xFF;
            h *= 1099511628211ull;
        }
    };
    for (snn_net* net : b->nets) {
        mix(net->N);
        mix(net->K);
        mix(net->D);
        mix((uint64_t)net->v.w_bf16 | (uint64_t)net->cfg.conn_rule << 8 | (uint64_t)net->v.n_bands << 16);
        mix((uint64_t)std::llround(net->cfg.imposed_rate_hz * 1000.0));
    }
    char key[320];
    std::string gpu(prop.name);
    for (char& ch : gpu)
        if (ch == ' ') ch = '_';
    snprintf(key, sizeof key, "batch:%s:%u:%016llx:%u", gpu.c_str(), n, (unsigned long long)h, trial_steps);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char k2[320];
            int m = 0, sh = 0;
            unsigned long long bud = 0;
            bool hit = false;
            while (fscanf(f, "%319s %d %d %llu", k2, &m, &sh, &bud) == 4)
                if (strcmp(k2, key) == 0) hit = true, b->mode = m, b->shape = sh, b->ring_budget = bud;
            fclose(f);
            if (hit) {
                snn_status st = snn_batch_set_ring_budget(b, b->ring_budget);
                if (st != SNN_OK) return st;
                if (mode_out) *mode_out = b->mode;
                if (shape_out) *shape_out = b->shape;
                if (budget_out) *budget_out = b->ring_budget;
                if (best_ms) *best_ms = -1.0;
                return SNN_OK;
            }
        }
    }
    // one snapshot of every network, restored after every trial; the trials
    // record no spikes (each raster counter parked at its capacity) and the
    // recorded rasters are kept
    std::vector<std::vector<char>> snap(n);
    std::vector<uint64_t> rcount(n);
    for (uint32_t i = 0; i < n; ++i) {
        size_t bytes = 0;
        snn_status st = snn_snapshot(b->nets[i], nullptr, 0, &bytes, stream);
        if (st != SNN_OK) return st;
        snap[i].resize(bytes);
        st = snn_snapshot(b->nets[i], snap[i].data(), bytes, &bytes, stream);
        if (st != SNN_OK) return st;
        DevState ds;
        std::memcpy(&ds, snap[i].data() + sizeof(SnapshotHeader), sizeof ds);
        rcount[i] = ds.raster_count;
    }
    auto restore = [&](bool last) -> snn_status {
        for (uint32_t i = 0; i < n; ++i) {
            snn_status st = snn_restore(b->nets[i], snap[i].data(), snap[i].size(), stream);
            if (st != SNN_OK) return st;
            CUDA_TRY(snn_set_raster_count(b->nets[i], last ? rcount[i] : b->nets[i]->v.raster_cap, s));
        }
        return SNN_OK;
    };
    if (snn_status st0 = restore(false); st0 != SNN_OK) return st0;
    const int32_t mode0 = b->mode, shape0 = b->shape;
    const uint64_t budget0 = b->ring_budget;
    const double fracs[] = {0.35, 0.5, 0.65};
    std::vector<uint32_t> warm(n, std::max(trial_steps / 4, 1u)), trial(n, trial_steps);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e300;
    int32_t bm = mode0, bs = shape0;
    uint64_t bb = budget0;
    std::vector<std::vector<uint64_t>> seen;
    snn_status st = SNN_OK;
    int cand = -1;
    for (int32_t m : {SNN_BATCH_GROUPS, SNN_BATCH_GLOBAL}) {
        for (int32_t sh : {0, 1}) {
            for (double fr : fracs) {
                ++cand;
                const uint64_t bud = l2 > 0 ? (uint64_t)(fr * l2) : (64ull << 20);
                b->mode = m;
                b->shape = sh;
                st = snn_batch_set_ring_budget(b, bud);
                if (st != SNN_OK) break;
                std::vector<uint64_t> plan;  // the waves (first, count, layout, shape) this candidate gives
                for (const BatchWave& w : b->waves)
                    plan.push_back((uint64_t)w.first | (uint64_t)w.count << 24 | (uint64_t)w.grouped << 48 |
                                   (uint64_t)(w.grouped ? 0 : w.shape) << 49);
                if (std::find(seen.begin(), seen.end(), plan) != seen.end()) continue;
                seen.push_back(plan);
                if ((st = snn_batch_step(b, warm.data(), stream)) != SNN_OK || (st = restore(false)) != SNN_OK) break;
                CUDA_TRY(cudaStreamSynchronize(s));
                CUDA_TRY(cudaEventRecord(e0, s));
                if ((st = snn_batch_step(b, trial.data(), stream)) != SNN_OK) break;
                CUDA_TRY(cudaEventRecord(e1, s));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.0f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if ((st = restore(false)) != SNN_OK) break;
                if (trial_ms) trial_ms[cand] = ms / trial_steps;
                if (ms < best) best = ms, bm = m, bs = sh, bb = bud;
            }
            if (st != SNN_OK) break;
        }
        if (st != SNN_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (snn_status st1 = restore(true); st == SNN_OK) st = st1;  // the rasters as they were
    if (st != SNN_OK) return st;
    b->mode = bm;
    b->shape = bs;
    st = snn_batch_set_ring_budget(b, bb);
    if (st != SNN_OK) return st;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %d %llu\n", key, (int)bm, (int)bs, (unsigned long long)bb);
            fclose(f);
        }
    }
    if (mode_out) *mode_out = bm;
    if (shape_out) *shape_out = bs;
    if (budget_out) *budget_out = bb;
    if (best_ms) *best_ms = best / trial_steps;
    return SNN_OK;
}

snn_status snn_batch_set_layout(snn_batch* b, int32_t mode, int32_t shape, uint64_t ring_budget) {
    if (!b || ring_budget == 0) return fail(SNN_EINVAL, "batch is NULL or the budget is 0");
    if (mode != SNN_BATCH_GLOBAL && mode != SNN_BATCH_GROUPS) return fail(SNN_EINVAL, "unknown batch mode %d", (int)mode);
    if (shape != 0 && shape != 1) return fail(SNN_EINVAL, "unknown batch shape %d", (int)shape);
    b->mode = mode;
    b->shape = shape;
    return snn_batch_set_ring_budget(b, ring_budget);
}

snn_status snn_batch_set_shape(snn_batch* b, int32_t shape) {
    if (!b) return fail(SNN_EINVAL, "batch is NULL");
    if (shape != 0 && shape != 1) return fail(SNN_EINVAL, "unknown batch shape %d", (int)shape);
    b->shape = shape;
    return snn_batch_set_ring_budget(b, b->ring_budget);
}

snn_status snn_batch_set_mode(snn_batch* b, int32_t mode) {
    if (!b) return fail(SNN_EINVAL, "batch is NULL");
    if (mode != SNN_BATCH_GLOBAL && mode != SNN_BATCH_GROUPS)
        return fail(SNN_EINVAL, "unknown batch mode %d", (int)mode);
    b->mode = mode;
    return snn_batch_set_ring_budget(b, b->ring_budget);
}

snn_status snn_plan_groups(const uint32_t* steps, const double* work, uint32_t n, uint32_t ctas, uint32_t* cta) {
    if (!steps || !work || !cta || n == 0) return fail(SNN_EINVAL, "steps, work and cta must be set and n > 0");
    if (n > ctas) return fail(SNN_EINVAL, "more networks (%u) than CTAs (%u)", n, ctas);
    for (uint32_t i = 0; i < n; ++i)
        if (!(work[i] >= 0.0) || !std::isfinite(work[i])) return fail(SNN_EINVAL, "work[%u] is not a finite value >= 0", i);
    std::vector<uint32_t> gcta(n + 1);
    partition_groups(steps, work, n, ctas, cta, gcta.data());
    return SNN_OK;
}

snn_status snn_plan_pull_bands(const snn_config* cfg, uint32_t sms, int32_t band_mode, uint32_t* bq,
                               uint32_t* run_ptr, uint32_t* runs, uint32_t cap, uint32_t* n_runs) {
    if (!cfg || !bq || !run_ptr || !n_runs) return fail(SNN_EINVAL, "cfg, bq, run_ptr and n_runs must be set");
    if (sms == 0) return fail(SNN_EINVAL, "sms must be at least 1");
    if (band_mode != 1 && band_mode != 2) return fail(SNN_EINVAL, "band_mode must be 1 or 2");
    if (cfg->grid_w == 0 || cfg->grid_h == 0 || cfg->neurons_per_module == 0)
        return fail(SNN_EINVAL, "empty grid");
    const uint64_t N64 = (uint64_t)cfg->grid_w * cfg->grid_h * cfg->neurons_per_module;
    if (N64 >= (1ull << 24)) return fail(SNN_EINVAL, "more than 2^24 neurons");
    const uint32_t N = (uint32_t)N64, M = cfg->neurons_per_module;
    bool all_entries = false;
    const std::vector<int16_t> off = pull_stencil(*cfg, &all_entries);
    const std::vector<uint32_t> b = pull_bands(N, M, (N + 3) / 4, sms, band_mode == 2);
    std::vector<uint2> r;
    std::vector<uint32_t> ptr;
    pull_build_runs(N, M, cfg->grid_w, cfg->grid_h, off, b, r, ptr, all_entries);
    std::copy(b.begin(), b.end(), bq);
    std::copy(ptr.begin(), ptr.end(), run_ptr);
    *n_runs = (uint32_t)r.size();
    if (r.size() > cap || (!runs && !r.empty()))
        return fail(SNN_EOVERFLOW, "%zu runs do not fit in %u", r.size(), cap);
    for (size_t i = 0; i < r.size(); ++i) {
        runs[2 * i] = r[i].x;
        runs[2 * i + 1] = r[i].y;
    }
    return SNN_OK;
}

snn_status snn_batch_groups(snn_batch* b, uint32_t* cta) {
    if (!b || !cta) return fail(SNN_EINVAL, "batch or cta is NULL");
    std::copy(b->last_cta.begin(), b->last_cta.end(), cta);
    return SNN_OK;
}

snn_status snn_batch_set_graph(snn_batch* b, int32_t enable) {
    if (!b) return fail(SNN_EINVAL, "batch is NULL");
    b->use_graph = enable != 0;
    return SNN_OK;
}

snn_status snn_batch_waves(snn_batch* b, uint32_t* waves, uint64_t* ring_budget) {
    if (!b) return fail(SNN_EINVAL, "batch is NULL");
    if (waves) *waves = (uint32_t)b->waves.size();
    if (ring_budget) *ring_budget = b->ring_budget;
    return SNN_OK;
}

snn_status snn_batch_step(snn_batch* b, const uint32_t* steps, void* stream) {
    if (!b || !steps) return fail(SNN_EINVAL, "batch or steps is NULL");
    NvtxRange range("snn_batch_step");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)b->nets.size();
    // the pinned staging buffer may still feed the previous call's copy
    CUDA_TRY(cudaStreamSynchronize(s));
    // the groups' times of the last call refine the work estimates
    for (uint32_t i = 0; i < n; ++i) {
        if (b->last_cta[i] == 0 || b->last_steps[i] == 0 || b->h_gns[i] == 0) continue;
        const double us = (double)b->h_gns[i] * 1e-3 / b->last_steps[i];
        b->work[i] = std::max(us - GROUP_FIXED_US, 0.05) * b->last_cta[i];
    }
    std::vector<uint32_t> key(b->waves.size(), 0);
    bool any = false;
    for (size_t k = 0; k < b->waves.size(); ++k) {
        const BatchWave& w = b->waves[k];
        for (uint32_t i = w.first; i < w.first + w.count; ++i) key[k] = std::max(key[k], steps[i]);
        any = any || key[k] > 0;
    }
    if (!any) return SNN_OK;
    std::copy(steps, steps + n, b->h_steps);
    std::fill(b->last_cta.begin(), b->last_cta.end(), 0u);
    for (size_t k = 0; k < b->waves.size(); ++k) {
        const BatchWave& w = b->waves[k];
        if (!w.grouped) continue;
        partition_groups(steps + w.first, b->work.data() + w.first, w.count, (uint32_t)w.grid,
                         b->last_cta.data() + w.first, b->h_steps + w.stage_off);
    }
    std::copy(steps, steps + n, b->last_steps.begin());
    CUDA_TRY(cudaMemcpyAsync(b->d_steps, b->h_steps, (size_t)b->stage_len * 4, cudaMemcpyHostToDevice, s));
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        for (size_t k = 0; k < b->waves.size(); ++k) {
            if (key[k] == 0) continue;
            const BatchWave& w = b->waves[k];
            cudaError_t e;
            if (w.count == 1) {
                // a network alone in its wave runs the single-network persistent kernel
                snn_net* net = b->nets[w.first];
                e = cudaMemsetAsync(&net->v.st->bar_count, 0, sizeof(uint32_t), q);
                if (e == cudaSuccess) e = launch_persistent(net->v, key[k], net->pgrid, q);
            } else if (w.grouped) {
                e = cudaSuccess;
                for (uint32_t i = w.first; i < w.first + w.count && e == cudaSuccess; ++i)
                    e = cudaMemsetAsync(&b->nets[i]->v.st->bar_count, 0, sizeof(uint32_t), q);
                if (e == cudaSuccess) e = launch_groups(w.gmeta, w.grid, q);
            } else {
                e = cudaMemsetAsync(&w.meta.bst->bar_count, 0, sizeof(uint32_t), q);
                if (e == cudaSuccess) e = launch_batch(w.meta, key[k], w.grid, w.shape, q);
            }
            if (e != cudaSuccess) return e;
        }
        // the groups' times, for the next call's partition
        return cudaMemcpyAsync(b->h_gns, b->d_gns, b->nets.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, q);
    };
    int slot = 0;
    snn_status st = timed_begin(b->ev, s, &slot);
    if (st != SNN_OK) return st;
    if (b->use_graph) {
        if (!b->graph_valid || b->graph_key != key) {
            if (b->exec) {
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
            if (!b->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
            CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t le = enqueue(b->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
            if (le != cudaSuccess || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return fail(SNN_ECUDA, "graph capture of the batch launches failed: %s",
                            cudaGetErrorString(le != cudaSuccess ? le : ce));
            }
            cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return fail(SNN_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
            b->graph_valid = true;
            b->graph_key = key;
        }
        CUDA_TRY(cudaGraphLaunch(b->exec, s));
    } else {
        CUDA_TRY(enqueue(s));
    }
    return timed_end(b->ev, s, slot);
}

snn_status snn_batch_time(snn_batch* b, double* ms, uint64_t* launches) {
    if (!b) return fail(SNN_EINVAL, "batch is NULL");
    snn_status st = drain(b->ev);
    if (st != SNN_OK) return st;
    if (ms) *ms = b->ev.total_ms;
    if (launches) *launches = b->ev.count;
    return SNN_OK;
}

void snn_batch_destroy(snn_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->h_steps) cudaFreeHost(b->h_steps);
    if (b->h_gns) cudaFreeHost(b->h_gns);
    destroy_events(b->ev);
    for (void* p : b->blocks) {
        if (b->free_fn)
            b->free_fn(p, b->alloc_ctx);
        else if (!b->alloc_fn)
            cudaFree(p);
    }
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Spatial decomposition (Sec. II-D, II-E; deferred arborization, Sec. II-C).

struct snn_shard {
    snn_net net;  // description, constants, allocator hook, device blocks
    uint32_t n_shards = 0, index = 0;
    uint32_t row0 = 0, row1 = 0, n0 = 0, n1 = 0, h0 = 0, h1 = 0, peer_lo = 0, peer_hi = 0;
    uint64_t nsyn = 0;
    uint32_t t = 0;  // next time step
    ShardView sv{};
};

namespace {

// Module rows of shard k of n: [H k / n, H (k + 1) / n).
uint32_t shard_row(uint32_t H, uint32_t n, uint32_t k) { return (uint32_t)((uint64_t)H * k / n); }

snn_status shard_build_impl(snn_shard* sh, cudaStream_t s) {
    snn_net* n = &sh->net;
    const snn_config& c = n->cfg;
    snn_status st = derive(n);
    if (st != SNN_OK) return st;
    uint32_t R2 = 0;
    std::vector<int16_t> off = disc_offsets(c, &R2);
    n->max_off = (uint32_t)(off.size() / 2);
    int R = 0;
    for (size_t o = 1; o < off.size(); o += 2) R = std::max(R, std::abs((int)off[o]));
    const uint32_t H = c.grid_h, WM = c.grid_w * c.neurons_per_module;
    sh->row0 = shard_row(H, sh->n_shards, sh->index);
    sh->row1 = shard_row(H, sh->n_shards, sh->index + 1);
    sh->n0 = sh->row0 * WM;
    sh->n1 = sh->row1 * WM;
    const uint32_t hr0 = (uint32_t)std::max(0, (int)sh->row0 - R);
    const uint32_t hr1 = std::min(H, sh->row1 + (uint32_t)R);
    sh->h0 = hr0 * WM;
    sh->h1 = hr1 * WM;
    // peers: the shards whose rows overlap the halo (this one included)
    sh->peer_lo = sh->n_shards;
    sh->peer_hi = 0;
    for (uint32_t k = 0; k < sh->n_shards; ++k)
        if (shard_row(H, sh->n_shards, k) < hr1 && shard_row(H, sh->n_shards, k + 1) > hr0) {
            sh->peer_lo = std::min(sh->peer_lo, k);
            sh->peer_hi = std::max(sh->peer_hi, k);
        }
    if (sh->peer_hi - sh->peer_lo + 1 > SHARD_MAX_LISTS)
        return fail(SNN_EINVAL, "shard %u reaches %u shards (at most %u)", sh->index, sh->peer_hi - sh->peer_lo + 1,
                    SHARD_MAX_LISTS);
    HostTables ht;
    host_tables(c, &ht);
    BuildView b{};
    fill_build_view(n, b);
    b.K = n->K;  // the fixed out-degree law
    b.Kpad = n->Kpad;
    std::vector<std::pair<void*, size_t>> temps;
    auto temp = [&](size_t bytes) -> void* {
        void* p = dev_alloc(n, bytes);
        if (p) temps.push_back({p, bytes});
        return p;
    };
    if (!ht.wtab.empty()) {
        float* wt = (float*)temp(ht.wtab.size() * 4);
        if (!wt) return fail(SNN_ENOMEM, "device allocation of the efficacy table failed");
        CUDA_TRY(cudaMemcpyAsync(wt, ht.wtab.data(), ht.wtab.size() * 4, cudaMemcpyHostToDevice, s));
        b.wtab = wt;
    }
    if (!ht.dthr.empty()) {
        uint64_t* dt = (uint64_t*)temp(ht.dthr.size() * 8);
        if (!dt) return fail(SNN_ENOMEM, "device allocation of the delay table failed");
        CUDA_TRY(cudaMemcpyAsync(dt, ht.dthr.data(), ht.dthr.size() * 8, cudaMemcpyHostToDevice, s));
        b.dthr = dt;
        b.n_dthr = (uint32_t)ht.dthr.size();
    }
    // the target-module tables of every source module (as snn_build_network builds them)
    const size_t tab = (size_t)n->n_modules * n->max_off;
    b.cdf_T = (uint32_t*)temp(tab * 4);
    b.cdf_mod = (uint32_t*)temp(tab * 4);
    b.cdf_n = (uint32_t*)temp((size_t)n->n_modules * 4);
    b.scratch = (double*)temp(tab * sizeof(double));
    int16_t* doff = (int16_t*)temp(off.size() * sizeof(int16_t));
    if (!b.cdf_T || !b.cdf_mod || !b.cdf_n || !b.scratch || !doff)
        return fail(SNN_ENOMEM, "device allocation of the construction tables failed");
    CUDA_TRY(cudaMemcpyAsync(doff, off.data(), off.size() * sizeof(int16_t), cudaMemcpyHostToDevice, s));
    b.offsets = doff;
    CUDA_TRY(launch_build_cdf(b, s));
    // the target-side table: halo rows restricted to the shard, counted then filled
    const uint32_t rows = sh->h1 - sh->h0;
    uint32_t* dcnt = (uint32_t*)temp((size_t)std::max<uint32_t>(rows, 1) * 4);
    uint64_t* rp = (uint64_t*)dev_alloc(n, ((size_t)rows + 1) * 8);
    if (!dcnt || !rp) return fail(SNN_ENOMEM, "device allocation of the shard table index failed");
    CUDA_TRY(launch_shard_count(b, sh->h0, rows, sh->n0, sh->n1, dcnt, s));
    std::vector<uint32_t> hc(rows);
    if (rows) CUDA_TRY(cudaMemcpyAsync(hc.data(), dcnt, (size_t)rows * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<uint64_t> hp((size_t)rows + 1, 0);
    for (uint32_t r = 0; r < rows; ++r) hp[r + 1] = hp[r] + hc[r];
    sh->nsyn = hp[rows];
    CUDA_TRY(cudaMemcpyAsync(rp, hp.data(), hp.size() * 8, cudaMemcpyHostToDevice, s));
    const size_t wbytes = n->v.w_bf16 ? 2 : 4;
    uint32_t* td = (uint32_t*)dev_alloc(n, std::max<uint64_t>(sh->nsyn, 1) * 4);
    void* w = dev_alloc(n, std::max<uint64_t>(sh->nsyn, 1) * wbytes);
    if (!td || !w) return fail(SNN_ENOMEM, "device allocation of %llu shard synapses failed",
                               (unsigned long long)sh->nsyn);
    CUDA_TRY(launch_shard_fill(b, sh->h0, rows, sh->n0, sh->n1, rp, td, w, s));
    // state, ring, outbox, raster, counters
    ShardView& sv = sh->sv;
    sv.n0 = sh->n0;
    sv.Nl = sh->n1 - sh->n0;
    sv.Nlpad = (sv.Nl + 255) / 256 * 256;
    sv.h0 = sh->h0;
    sv.rows = rows;
    sv.row_ptr = rp;
    sv.td = td;
    sv.w = w;
    const size_t Np = std::max<uint32_t>(sv.Nlpad, 256);
    sv.V = (float*)dev_alloc(n, Np * 4);
    sv.c = (float*)dev_alloc(n, Np * 4);
    sv.ref = (uint8_t*)dev_alloc(n, Np);
    sv.ring = (int32_t*)dev_alloc(n, (size_t)n->D * Np * 4);
    sv.spk_bits = (uint32_t*)dev_alloc(n, Np / 32 * 4);
    sv.out_ids = (uint32_t*)dev_alloc(n, Np * 4);
    sv.out_cnt = (uint32_t*)dev_alloc(n, 4);
    const uint64_t cap = c.raster_capacity ? c.raster_capacity : 1;
    sv.raster_t = (uint32_t*)dev_alloc(n, cap * 4);
    sv.raster_id = (uint32_t*)dev_alloc(n, cap * 4);
    sv.raster_cap = c.raster_capacity;
    sv.cnt = (ShardCounters*)dev_alloc(n, sizeof(ShardCounters));
    if (!sv.V || !sv.c || !sv.ref || !sv.ring || !sv.spk_bits || !sv.out_ids || !sv.out_cnt || !sv.raster_t ||
        !sv.raster_id || !sv.cnt)
        return fail(SNN_ENOMEM, "device allocation of the shard state failed");
    CUDA_TRY(launch_shard_init(b, sh->n0, sv.Nl, sv.V, sv.c, sv.ref, s));
    CUDA_TRY(cudaMemsetAsync(sv.ring, 0, (size_t)n->D * Np * 4, s));
    CUDA_TRY(cudaMemsetAsync(sv.out_cnt, 0, 4, s));
    CUDA_TRY(cudaMemsetAsync(sv.cnt, 0, sizeof(ShardCounters), s));
    CUDA_TRY(cudaStreamSynchronize(s));  // the construction buffers are released next
    for (auto& tb : temps) free_block(n, tb.first, tb.second);
    return SNN_OK;
}

}  // namespace

extern "C" {

snn_status snn_shard_build(const snn_config* cfg, uint32_t n_shards, uint32_t index, snn_alloc_fn alloc_fn,
                           snn_free_fn free_fn, void* alloc_ctx, void* stream, snn_shard** out) {
    if (!out) return fail(SNN_EINVAL, "out is NULL");
    *out = nullptr;
    snn_status st = validate(cfg);
    if (st != SNN_OK) return st;
    if (cfg->conn_rule != SNN_RULE_FIXED_K)
        return fail(SNN_EINVAL, "shards are built for the fixed out-degree rule (conn_rule = SNN_RULE_FIXED_K)");
    if (cfg->stdp) return fail(SNN_EINVAL, "shards run static synapses (stdp = 0)");
    if (n_shards == 0 || index >= n_shards || n_shards > cfg->grid_h)
        return fail(SNN_EINVAL, "need 0 <= index < n_shards <= grid_h (got %u of %u, grid_h %u)", index, n_shards,
                    cfg->grid_h);
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return fail(SNN_EINVAL, "alloc_fn and free_fn must both be set or both be NULL");
    snn_shard* sh = new (std::nothrow) snn_shard();
    if (!sh) return fail(SNN_ENOMEM, "host allocation failed");
    sh->net.cfg = *cfg;
    sh->net.alloc_fn = alloc_fn;
    sh->net.free_fn = free_fn;
    sh->net.alloc_ctx = alloc_ctx;
    cudaGetDevice(&sh->net.device);
    sh->n_shards = n_shards;
    sh->index = index;
    NvtxRange range("snn_shard_build");
    st = shard_build_impl(sh, (cudaStream_t)stream);
    if (st != SNN_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        release_all(&sh->net);
        delete sh;
        return st;
    }
    *out = sh;
    return SNN_OK;
}

snn_status snn_shard_info(snn_shard* sh, snn_shard_info_t* out) {
    if (!sh || !out) return fail(SNN_EINVAL, "shard or out is NULL");
    out->n_shards = sh->n_shards;
    out->index = sh->index;
    out->row0 = sh->row0;
    out->row1 = sh->row1;
    out->n0 = sh->n0;
    out->n1 = sh->n1;
    out->h0 = sh->h0;
    out->h1 = sh->h1;
    out->peer_lo = sh->peer_lo;
    out->peer_hi = sh->peer_hi;
    out->D = sh->net.D;
    out->table_synapses = sh->nsyn;
    out->device_bytes = sh->net.device_bytes;
    out->t = sh->t;
    return SNN_OK;
}

snn_status snn_shard_integrate(snn_shard* sh, void* stream) {
    if (!sh) return fail(SNN_EINVAL, "shard is NULL");
    CUDA_TRY(launch_shard_step(sh->net.v, sh->sv, sh->t, (cudaStream_t)stream));
    return SNN_OK;
}

snn_status snn_shard_outbox(snn_shard* sh, uint32_t** ids, uint32_t** count) {
    if (!sh || !ids || !count) return fail(SNN_EINVAL, "shard, ids or count is NULL");
    *ids = sh->sv.out_ids;
    *count = sh->sv.out_cnt;
    return SNN_OK;
}

snn_status snn_shard_deliver(snn_shard* sh, const uint32_t* const* ids, const uint32_t* const* counts,
                             uint32_t n_lists, void* stream) {
    if (!sh) return fail(SNN_EINVAL, "shard is NULL");
    if (n_lists > SHARD_MAX_LISTS || (n_lists && (!ids || !counts)))
        return fail(SNN_EINVAL, "at most %u inbound lists, with ids and counts", SHARD_MAX_LISTS);
    ShardInbound in{};
    for (uint32_t l = 0; l < n_lists; ++l) {
        if (!ids[l] || !counts[l]) return fail(SNN_EINVAL, "inbound list %u is NULL", l);
        in.ids[l] = ids[l];
        in.cnt[l] = counts[l];
    }
    in.n = n_lists;
    CUDA_TRY(launch_shard_deliver(sh->net.v, sh->sv, in, sh->t, (cudaStream_t)stream));
    sh->t += 1;
    return SNN_OK;
}

snn_status snn_shards_run(snn_shard* const* shards, uint32_t n, uint32_t n_steps, void* stream) {
    if (!shards || n == 0) return fail(SNN_EINVAL, "no shards");
    for (uint32_t k = 0; k < n; ++k) {
        if (!shards[k] || shards[k]->n_shards != n || shards[k]->index != k)
            return fail(SNN_EINVAL, "shards must be indexes 0..%u of one %u-way decomposition, in order", n - 1, n);
        if (shards[k]->t != shards[0]->t) return fail(SNN_EINVAL, "shards are at different time steps");
        if (memcmp(&shards[k]->net.cfg, &shards[0]->net.cfg, sizeof(snn_config)) != 0)
            return fail(SNN_EINVAL, "shards of different network descriptions");
    }
    NvtxRange range("snn_shards_run");
    for (uint32_t step = 0; step < n_steps; ++step) {
        for (uint32_t k = 0; k < n; ++k) {
            snn_status st = snn_shard_integrate(shards[k], stream);
            if (st != SNN_OK) return st;
        }
        // one device: the exchange is the peers' outboxes read in place
        for (uint32_t k = 0; k < n; ++k) {
            const uint32_t* ids[SHARD_MAX_LISTS];
            const uint32_t* cnt[SHARD_MAX_LISTS];
            uint32_t m = 0;
            for (uint32_t q = shards[k]->peer_lo; q <= shards[k]->peer_hi; ++q, ++m) {
                ids[m] = shards[q]->sv.out_ids;
                cnt[m] = shards[q]->sv.out_cnt;
            }
            snn_status st = snn_shard_deliver(shards[k], ids, cnt, m, stream);
            if (st != SNN_OK) return st;
        }
    }
    return SNN_OK;
}

snn_status snn_shard_read_spikes(snn_shard* sh, uint32_t* steps, uint32_t* ids, size_t cap, size_t* n_out,
                                 void* stream) {
    if (!sh || !n_out) return fail(SNN_EINVAL, "shard or n_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    ShardCounters hc;
    CUDA_TRY(cudaMemcpyAsync(&hc, sh->sv.cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    uint64_t avail = std::min<uint64_t>(hc.raster_count, sh->sv.raster_cap);
    const size_t k = (size_t)std::min<uint64_t>(avail, cap);
    if (k && steps) CUDA_TRY(cudaMemcpyAsync(steps, sh->sv.raster_t, k * 4, cudaMemcpyDeviceToHost, s));
    if (k && ids) CUDA_TRY(cudaMemcpyAsync(ids, sh->sv.raster_id, k * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *n_out = k;
    if (hc.raster_count > sh->sv.raster_cap) return fail(SNN_EOVERFLOW, "shard raster overflowed");
    return SNN_OK;
}

snn_status snn_shard_get_state(snn_shard* sh, float* V, float* c, uint8_t* ref, int32_t* ring, void* stream) {
    if (!sh) return fail(SNN_EINVAL, "shard is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const ShardView& sv = sh->sv;
    if (V) CUDA_TRY(cudaMemcpyAsync(V, sv.V, (size_t)sv.Nl * 4, cudaMemcpyDeviceToHost, s));
    if (c) CUDA_TRY(cudaMemcpyAsync(c, sv.c, (size_t)sv.Nl * 4, cudaMemcpyDeviceToHost, s));
    if (ref) CUDA_TRY(cudaMemcpyAsync(ref, sv.ref, sv.Nl, cudaMemcpyDeviceToHost, s));
    if (ring)
        CUDA_TRY(cudaMemcpy2DAsync(ring, (size_t)sv.Nl * 4, sv.ring, (size_t)sv.Nlpad * 4, (size_t)sv.Nl * 4,
                                   sh->net.D, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_shard_stats(snn_shard* sh, snn_stats* out, void* stream) {
    if (!sh || !out) return fail(SNN_EINVAL, "shard or out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    ShardCounters hc;
    CUDA_TRY(cudaMemcpyAsync(&hc, sh->sv.cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    memset(out, 0, sizeof *out);
    out->steps = sh->t;
    out->n_spikes = hc.n_spikes;
    out->rec_events = hc.rec_events;
    out->ext_events = hc.ext_events;
    out->raster_count = hc.raster_count;
    out->raster_capacity = sh->sv.raster_cap;
    return SNN_OK;
}

void snn_shard_destroy(snn_shard* sh) {
    if (!sh) return;
    cudaDeviceSynchronize();
    release_all(&sh->net);
    delete sh;
}

}  // extern "C"
